"""Pure-Python twin of the schoolbook oracle, for tiny inputs -- TEST INFRASTRUCTURE ONLY.

Computes the definition of the product in Z[x] (Harvey, Sec. 3) with Python's
arbitrary-precision integers: h_k = sum over i + j = k of f_i g_j.
"""
from __future__ import annotations


def poly_mul(f: list[int], g: list[int]) -> list[int]:
    """h = f g for coefficient lists (index = exponent); any signs, any sizes."""
    if not f or not g:
        raise ValueError("polynomials need length >= 1")
    h = [0] * (len(f) + len(g) - 1)
    for i, fi in enumerate(f):
        for j, gj in enumerate(g):
            h[i + j] += fi * gj
    return h


def poly_eval(f: list[int], x: int) -> int:
    """f(x) by direct summation of f_i x^i."""
    return sum(c * x ** i for i, c in enumerate(f))


def poly_mul_mod(f: list[int], g: list[int], p: int) -> list[int]:
    """h mod p, coefficientwise, for the (Z/pZ)[x] application of Sec. 4."""
    return [c % p for c in poly_mul(f, g)]


def biv_mul_mod(f: list[list[int]], g: list[list[int]], p: int) -> list[list[int]]:
    """h = f g in (Z/pZ)[x, y] for coefficient arrays f[i][j] (the coefficient
    of x^j y^i), by the plain double convolution (Sec. 2's setting)."""
    ly, lx = len(f), len(f[0])
    h = [[0] * (2 * lx - 1) for _ in range(2 * ly - 1)]
    for i in range(ly):
        for j in range(lx):
            for i2 in range(len(g)):
                for j2 in range(len(g[0])):
                    h[i + i2][j + j2] += f[i][j] * g[i2][j2]
    return [[c % p for c in row] for row in h]
