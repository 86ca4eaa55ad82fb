"""Failure handling that needs no GPU: a corrupt, truncated or mis-keyed
dispatch state is refused (the library keeps its built-in choice), and the
host-side hooks and status calls exist in the C ABI."""
import json
import os
import shutil

import pytest

from paper_0712_4046_gb300 import dispatch


@pytest.fixture()
def state(tmp_path):
    if not os.path.exists(dispatch.STATE_FILE):
        pytest.skip("no committed dispatch state")
    p = tmp_path / "state.json"
    shutil.copy(dispatch.STATE_FILE, p)
    return p


def test_committed_state_verifies(state):
    body = dispatch.load_state(str(state))
    assert body is not None and body["format"] == dispatch.FORMAT
    assert body["table"] and body["mlp"]


def test_corrupt_state_is_refused(state, monkeypatch):
    doc = json.loads(state.read_text())
    doc["body"]["table"][0][4] = 5 - doc["body"]["table"][0][4]   # one choice changed
    state.write_text(json.dumps(doc))
    assert dispatch.load_state(str(state)) is None
    calls = []
    import paper_0712_4046_gb300 as ks
    monkeypatch.setattr(ks, "dispatch_set_table", lambda rows: calls.append(rows))
    assert dispatch.install(str(state)) is False
    assert calls == []


def test_truncated_and_missing_state_are_refused(state, tmp_path):
    text = state.read_text()
    state.write_text(text[: len(text) // 2])
    assert dispatch.load_state(str(state)) is None
    assert dispatch.load_state(str(tmp_path / "absent.json")) is None


def test_mis_keyed_state_is_refused(state, monkeypatch):
    body = dispatch.load_state(str(state))
    other = dict(body["key"], device="some other GPU", sms=body["key"]["sms"] + 1)
    monkeypatch.setattr(dispatch, "device_key", lambda: other)
    calls = []
    import paper_0712_4046_gb300 as ks
    monkeypatch.setattr(ks, "dispatch_set_table", lambda rows: calls.append(rows))
    monkeypatch.setattr(ks, "mlp_set_params", lambda p: calls.append(p))
    assert dispatch.install(str(state)) is False
    assert calls == []


def test_fault_hooks_are_exported():
    import paper_0712_4046_gb300 as ks
    for name in ("ks_debug_fail_allocs", "ks_debug_tc_stall", "ks_plan_status",
                 "ks_status_sync"):
        assert hasattr(ks.lib, name)
    assert ks.lib.ks_plan_status(None) == ks.KS_EINVAL
    ks.debug_fail_allocs(0)
    ks.debug_tc_stall(False, 0)
