"""The C ABI without a GPU: the library loads, exports every function that
``include/*.h`` declares, and its host-only planning calls give the sizes of
Sec. 3 (N per variant, output limbs)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ks():
    import __graft_entry__ as ge
    ge.build()
    import paper_0712_4046_gb300 as ks
    return ks


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            if name.startswith("ks_") and not name.endswith("_t"):
                names.add(name)
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ks_mul", "ks_mul_ex", "ks_mul_host", "ks_mul_mod", "ks_mul_batch",
                 "ks_out_limbs", "ks_workspace_bytes", "ks_status_sync", "ks_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(ks):
    lib = ctypes.CDLL(ks._LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_eval_bits_follow_the_paper(ks):
    # N = 2b + e, b + ceil(e/2), b + ceil(e/2), ceil((2b + e)/4)  (Sec. 3.1-3.4)
    for L, b in [(1, 1), (4, 3), (1024, 64), (16384, 48), (1 << 20, 256), (1000, 7)]:
        e = (L - 1).bit_length()
        assert ks.eval_bits(L, L, b, 1) == 2 * b + e
        assert ks.eval_bits(L, L, b, 2) == b + (e + 1) // 2
        assert ks.eval_bits(L, L, b, 3) == b + (e + 1) // 2
        assert ks.eval_bits(L, L, b, 4) == (2 * b + e + 3) // 4
    # config sizes quoted from the Propositions: L=16384, b=48 -> KS1 N=110
    assert ks.eval_bits(16384, 16384, 48, 1) == 110
    assert ks.eval_bits(16384, 16384, 48, 4) == 28
    assert ks.eval_bits(1024, 1024, 64, 4) == 35
    # unequal lengths take e from the shorter polynomial
    assert ks.eval_bits(5, 1000, 10, 1) == 2 * 10 + 3


def test_unequal_sizes_plan_with_bf_plus_bg(ks):
    # Sec. 3.1-3.4 with bf + bg in place of 2b: the plan's N is the step model's
    # (pinned there against the plain product and its tightness), and it is below
    # the equal-size N at max(bf, bg) whenever the sizes differ
    from oracle import ks_steps as S
    shapes = [(300, 200, 48, 16), (100, 150, 130, 20), (1, 700, 5, 200), (500, 1, 3, 1),
              (16384, 16384, 4, 60), (1024, 4096, 1, 64), (2000, 3000, 4, 4), (64, 64, 64, 65)]
    for lf, lg, bf, bg in shapes:
        e = S.ceil_log(min(lf, lg), 2)
        for sg in (False, True):
            for v in (1, 2, 3, 4):
                info = ks.plan_info(lf, lg, bf, sg, v, ks.ENGINE_NTT, bits_g=bg)
                want = S.signed_N(v, bf, bg, e) if sg else S.variant_N_bits(v, bf, bg, e)
                assert info["N"] == want, (lf, lg, bf, bg, sg, v)
                ol = (bf + bg + e + int(sg) + 63) // 64
                assert info["out_limbs"] == ks.out_limbs_bits(lf, lg, bf, bg, sg) == ol
                assert info["in_limbs"] == (max(bf, bg) + 63) // 64
                if bf != bg and v == 1:
                    eq = ks.plan_info(lf, lg, max(bf, bg), sg, v, ks.ENGINE_NTT)
                    assert info["N"] < eq["N"]
            # equal sizes: the same plan as ks_plan_info
            assert ks.plan_info(lf, lg, bf, sg, 4, ks.ENGINE_NTT, bits_g=bf) == \
                ks.plan_info(lf, lg, bf, sg, 4, ks.ENGINE_NTT)
    with pytest.raises(ks.KSError):
        ks.out_limbs_bits(5, 5, 8, 0, False)
    with pytest.raises(ks.KSError):
        ks.plan_info(5, 5, 8, False, 1, ks.ENGINE_NTT, bits_g=2049)


def test_out_limbs_and_errors(ks):
    assert ks.out_limbs(1024, 1024, 64, False) == 3     # 138 bits
    assert ks.out_limbs(16384, 16384, 48, True) == 2    # 111 bits
    assert ks.out_limbs(1, 1, 32, False) == 1
    with pytest.raises(ks.KSError):
        ks.out_limbs(0, 5, 8, False)
    with pytest.raises(ks.KSError):
        ks.out_limbs(5, 5, 0, False)
    with pytest.raises(ks.KSError):
        ks.eval_bits(5, 5, 8, 7)
    assert ks.lib.ks_strerror(ks.KS_EINVAL) == b"invalid argument"
    assert ks.lib.ks_version() >= 100


def test_workspace_is_host_computable(ks):
    for v in (1, 2, 3, 4):
        n = ks.workspace_bytes(16384, 16384, 48, True, v, ks.ENGINE_SCHOOLBOOK)
        assert n > 0 and n % 256 == 0
    v, e = ks.choose(16384, 16384, 48, True)
    assert v in (1, 2, 3, 4) and e in (1, 2, 3)


def test_binding_refuses_wrong_layouts_before_any_device_call():
    # shapes, dtypes and devices are checked before a pointer reaches the C ABI
    import torch

    import paper_0712_4046_gb300 as ks
    lf, lg, b = 5, 4, 70  # two limbs per coefficient
    ol = ks.out_limbs(lf, lg, b, True)
    f = torch.zeros((lf, 2), dtype=torch.int64)
    g = torch.zeros((lg, 2), dtype=torch.int64)
    h = torch.zeros((lf + lg - 1, ol), dtype=torch.int64)
    bad = [
        (h, torch.zeros((lf, 1), dtype=torch.int64), g, "shape"),          # one limb short
        (h, f, torch.zeros((lg, 2), dtype=torch.int32), "dtype"),          # 4-byte elements
        (torch.zeros((lf + lg, ol), dtype=torch.int64), f, g, "shape"),   # h one row long
        (torch.zeros((lf + lg - 1, ol + 1), dtype=torch.int64), f, g, "shape"),
        (h, torch.zeros((2, lf), dtype=torch.int64).t(), g, "contiguous"),  # transposed
        (h, torch.zeros((lf, 2, 1), dtype=torch.int64), g, "2-d"),
        (h, torch.zeros((lf, 4), dtype=torch.int64)[:, ::2], g, "contiguous"),
    ]
    for hh, ff, gg, what in bad:
        with pytest.raises(ValueError, match=what):
            ks.ks_mul(hh, ff, gg, b, True, ks.KS_4)
    # correct layouts on the host: refused for the device, still before the ABI
    with pytest.raises(ValueError, match="CUDA"):
        ks.ks_mul(h, f, g, b, True, ks.KS_4)
    with pytest.raises(ValueError, match="CUDA"):
        ks.ks_mul_static(h, f, g, b, True, ks.KS_4)
    with pytest.raises(ValueError, match="shape"):
        ks.ks_mul_bits(h, f, 70, torch.zeros((lg, 2), dtype=torch.int64), 64, True)
    with pytest.raises(ValueError, match="shape"):
        ks.ks_mul_mod(torch.zeros((lf + lg - 1, 2), dtype=torch.int64),
                      torch.zeros((lf, 1), dtype=torch.int64),
                      torch.zeros((lg, 1), dtype=torch.int64), 97)


def _tile_offsets(dmax, R):
    """Block offsets of each output tile of one sub-product (tile t meets the
    offsets max(0, 128 t - R + 1) .. min(128 t + 127, dmax))."""
    T = (dmax + R + 127) // 128
    return [min(128 * t + 127, dmax) - max(0, 128 * t - R + 1) + 1 for t in range(T)]


@pytest.mark.parametrize("shape", [(16384, 16384, 48, True, 4), (2500, 2300, 48, True, 1),
                                   (4000, 1000, 20, False, 3), (65536, 65536, 8, False, 2)])
@pytest.mark.parametrize("grid", [152, 37])
def test_tensor_core_split(ks, shape, grid):
    # the host's split of the tensor-core work: it covers every offset once, in
    # order; each CTA's first item is the tile holding its first offset; a share
    # that runs into a further tile is charged two offsets, and with that charge
    # the shares cost the same to within the charge and the rounding
    lf, lg, b, sg, v = shape
    info = ks.plan_info(lf, lg, b, sg, v, ks.ENGINE_TC)
    sp = ks.tc_split(lf, lg, b, sg, v, grid)
    dmax, R = (info["nA"] + 126) // 128, (info["nB"] + 127) // 128
    per_tile = _tile_offsets(dmax, R)
    starts, tiles = [], []  # every tile's first position, with (q, t)
    pos = 0
    for q in range(info["nprod"]):
        for t, n in enumerate(per_tile):
            starts.append(pos)
            tiles.append((q, t))
            pos += n
    assert sp["total"] == pos
    at = sp["at"]
    assert at[0] == 0 and at[-1] == pos
    assert all(x <= y for x, y in zip(at, at[1:]))
    import bisect
    costs = []
    for k in range(grid):
        if at[k] < pos:
            j = bisect.bisect_right(starts, at[k]) - 1
            assert (sp["first_q"][k], sp["first_tile"][k]) == tiles[j], k
        inside = sum(1 for s in starts if at[k] < s < at[k + 1])
        costs.append(at[k + 1] - at[k] + 2 * inside)
    V = pos + 2 * (len(starts) - 1)
    assert max(costs) <= V / grid + 2 + 1, (max(costs), V / grid)


def test_tensor_core_split_edges(ks):
    # one coefficient each: a single tile with two offsets; more CTAs than
    # offsets leave the extra shares empty; a long thin product stays ordered
    sp = ks.tc_split(1, 1, 1, False, 1, 1)
    assert sp["at"] == [0, sp["total"]] and sp["first_tile"] == [0]
    sp = ks.tc_split(1, 1, 1, False, 1, 152)
    assert sp["at"][0] == 0 and sp["at"][-1] == sp["total"]
    assert all(x <= y for x, y in zip(sp["at"], sp["at"][1:]))
    sp = ks.tc_split(3, 200000, 8, True, 4, 152)
    assert sp["at"][-1] == sp["total"] and all(x <= y for x, y in zip(sp["at"], sp["at"][1:]))
    with pytest.raises(ks.KSError):
        ks.tc_split(100, 100, 8, False, 1, 161)  # more CTAs than the split holds


def test_binding_checks_unequal_size_layouts():
    # ks_mul_bits: f and g with their own limb counts, h with the limbs of
    # bf + bg (not of 2 max(bf, bg)); plan problems with coeff_bits_g likewise
    import torch

    import paper_0712_4046_gb300 as ks
    lf, lg, bf, bg = 40, 30, 130, 20
    ol = ks.out_limbs_bits(lf, lg, bf, bg, True)
    assert ol < ks.out_limbs(lf, lg, max(bf, bg), True)
    f = torch.zeros((lf, 3), dtype=torch.int64)
    g = torch.zeros((lg, 1), dtype=torch.int64)
    with pytest.raises(ValueError, match="shape"):  # h sized for 2 max(bf, bg)
        ks.ks_mul_bits(torch.zeros((lf + lg - 1, ks.out_limbs(lf, lg, bf, True)),
                                   dtype=torch.int64), f, bf, g, bg, True)
    with pytest.raises(ValueError, match="shape"):  # g with f's limb count
        ks.ks_mul_bits(torch.zeros((lf + lg - 1, ol), dtype=torch.int64), f, bf,
                       torch.zeros((lg, 3), dtype=torch.int64), bg, True)
    with pytest.raises(ValueError, match="CUDA"):  # right layouts, host tensors
        ks.ks_mul_bits(torch.zeros((lf + lg - 1, ol), dtype=torch.int64), f, bf, g, bg, True)
    with pytest.raises(ValueError, match="shape"):
        ks.Plan([dict(h=torch.zeros((lf + lg - 1, ol), dtype=torch.int64), f=f,
                      g=torch.zeros((lg, 3), dtype=torch.int64), coeff_bits=bf,
                      coeff_bits_g=bg, is_signed=True)])
