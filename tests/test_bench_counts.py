"""The work counts bench.py reports rooflines against, checked by brute force on small shapes.

eri_products: the emulated ERI multiplies only the rows (x, y), x <= y, of L^T (L^P symmetric);
row (x, y) stores to V_xb (x in the block's a range, b >= x) and V_yb (y in the a range, x < y,
b >= y); a product is needed when one of them is.  ladder_products: the ladder's row-column
products over the a <= b pairs in the plain and symmetric/antisymmetric forms.
"""
import itertools

import pytest

from bench import eri_products, ladder_products


def blocks(nv, n_a, n_b):
    for b0 in range(0, nv, n_b):
        for a0 in range(0, nv, n_a):
            a1, b1 = min(nv, a0 + n_a), min(nv, b0 + n_b)
            if a0 <= b1 - 1:
                yield a0, a1, b0, b1


def brute_eri(nv, n_a, n_b):
    total = 0
    for a0, a1, b0, b1 in blocks(nv, n_a, n_b):
        for x, y in itertools.product(range(nv), repeat=2):
            if x > y:
                continue
            direct = a0 <= x < a1
            mirror = x < y and a0 <= y < a1
            for b in range(b0, b1):
                if (direct and b >= x) or (mirror and b >= y):
                    total += nv   # every d of the column block
    return total


@pytest.mark.parametrize("nv,n_a,n_b", [(1, 1, 1), (5, 5, 5), (7, 3, 2), (9, 9, 4), (11, 4, 11), (13, 5, 3)])
def test_eri_products_brute_force(nv, n_a, n_b):
    assert eri_products(nv, n_a, n_b) == brute_eri(nv, n_a, n_b)


def test_eri_products_cover_every_needed_entry_once():
    # every V entry (a <= b, c, d) comes from exactly one computed product: the row
    # (min(a, c), max(a, c)) and the column (b, d)
    nv = 6
    seen = {}
    for x, y in itertools.product(range(nv), repeat=2):
        if x > y:
            continue
        for b, d in itertools.product(range(nv), repeat=2):
            if b >= x:
                seen.setdefault((x, b, y, d), []).append((x, y, b, d))
            if x < y and b >= y:
                seen.setdefault((y, b, x, d), []).append((x, y, b, d))
    need = {(a, b, c, d) for a, b, c, d in itertools.product(range(nv), repeat=4) if a <= b}
    assert set(seen) == need
    assert all(len(v) == 1 for v in seen.values())
    assert eri_products(nv, nv, nv) == len({v[0] for v in seen.values()}) * 1


def test_single_block_closed_form():
    for nv in (1, 2, 17, 64):
        assert eri_products(nv, nv, nv) == nv * nv * (nv + 1) * (2 * nv + 1) // 6


@pytest.mark.parametrize("no,nv", [(1, 1), (2, 3), (4, 5)])
def test_ladder_products_brute_force(no, nv):
    pairs = [(a, b) for a in range(nv) for b in range(nv) if a <= b]
    plain = sum(1 for _ in pairs for _ in range(no * no) for _ in range(nv * nv))
    assert ladder_products(no, nv, "plain") == plain
    pm = 0
    for _ in pairs:
        pm += sum(1 for i in range(no) for j in range(no) if i <= j) * sum(1 for c in range(nv) for d in range(nv) if c <= d)
        pm += sum(1 for i in range(no) for j in range(no) if i < j) * sum(1 for c in range(nv) for d in range(nv) if c < d)
    assert ladder_products(no, nv, "pm") == pm


def test_fp64_roofline_counts_the_kernel_that_carries_the_flops():
    # the fused kernel carries the whole call's packed flops; the rebuild order's ERI kernel its
    # 2 X v^2 p share (timed separately from the ladder)
    import types
    import bench
    import paper_2603_20912_gb300 as lad
    from paper_2603_20912_gb300 import build
    build.build()
    cfg = types.SimpleNamespace(no=20, nv=400, nchol=1260)
    kms = {"fused": 2000.0, "eri": 1500.0}
    p = 400 * 401 // 2
    for path, flops, ms in [(lad.LADDER_PATH_FUSED, lad.ladder_flops(20, 400, 1260), 2000.0),
                            (lad.LADDER_PATH_ERI, 2.0 * 1260 * 400 * 400 * p, 1500.0)]:
        plan = types.SimpleNamespace(path=lambda path=path: path)
        r = bench.fp64_roofline(lad, plan, cfg, kms, 2, 1.1)
        assert r["achieved"] == pytest.approx(flops * 2 / (ms * 1e-3) / 1e12)
        assert r["frac"] == pytest.approx(r["achieved"] / 1.1)
    assert "fused" in bench.fp64_roofline(lad, types.SimpleNamespace(path=lambda: 2), cfg, kms, 1, 1.1)["kernel"]


def test_traffic_is_reported_only_for_the_captured_sources_and_blocking(monkeypatch):
    import bench
    sha, nbytes, src, blocking = bench.TRAFFIC_CAPTURES[("emu", "c3")]
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)
    assert bench.captured_traffic("emu", "c3", blocking) == (nbytes, src)
    assert bench.captured_traffic("emu", "c3", (blocking[0], blocking[1] + 1)) == (None, None)
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: "0" * 16)
    assert bench.captured_traffic("emu", "c3", blocking) == (None, None)
    assert bench.captured_traffic("emu", "c9", blocking) == (None, None)
