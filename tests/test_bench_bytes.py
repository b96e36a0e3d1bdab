"""The roofline of bench.py.  Its numerator (the method's bytes of the opacity stage) against a count
made from the oracle's layer profile: every distinct (molecule, P row, T row) table row that
the layers' bilinear brackets touch (Sec. 5: the largest grid node at or below the layer's
pressure and temperature, clamped to the grid), the CIA rows of the temperature brackets, one
Rayleigh row per species and the FP64 native output.  bench.py computes the layer pressures
and temperatures itself; the oracle's profile and a brute-force bracket search check them."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def bracket_brute(grid, v):
    """Largest i <= len(grid) - 2 with grid[i] <= v (v clamped to the grid), by a scan."""
    v = min(max(v, grid[0]), grid[-1])
    i = 0
    for k in range(len(grid) - 1):
        if grid[k] <= v:
            i = k
    return i


def method_bytes_from_profile(tb, P, T):
    W = tb.n_wn
    rows = set()
    for p, t in zip(P, T):
        a, b = bracket_brute(tb.p_grid, p), bracket_brute(tb.t_grid, t)
        rows |= {(a, b), (a, b + 1), (a + 1, b), (a + 1, b + 1)}
    by = tb.sigma.shape[0] * len(rows) * W * 4
    if tb.cia_pair.shape[0]:
        tc = set()
        for t in T:
            c = bracket_brute(tb.t_grid_cia, t)
            tc |= {c, c + 1}
        by += tb.cia_pair.shape[0] * len(tc) * W * 4
    if tb.rayleigh is not None:
        by += len(tb.species) * W * 4
    return by + W * 8, len(rows)


@pytest.mark.parametrize("n_wn", [1000, 2003])
def test_method_bytes_match_oracle_profile(n_wn):
    import bench
    from oracle import oracle as O
    from paper_1912_07759_gb300 import synthetic as S
    tb = S.make_tables(2, 5, 22, 27, n_wn, with_cia=True)
    atm = S.config2_atmosphere()
    prof = O.profile(tb, atm)
    want, n_rows = method_bytes_from_profile(tb, prof["P"], prof["T"])
    assert n_rows > 4                       # the 4-node profile crosses several (P, T) cells
    assert bench.algorithmic_bytes(tb, atm) == want
    # the two-stage design adds exactly the K write, N layers x W x 4 bytes
    assert bench.algorithmic_bytes(tb, atm, "design_opacity") == want + atm.n_layers * n_wn * 4


def test_method_bytes_of_the_full_size_workload():
    """At 200,000 wavenumbers the count is 292.8 MB: 65 distinct (P, T) rows of 5 absorbers
    (260 MB), 16 CIA temperature rows of 2 pairs (25.6 MB), 7 Rayleigh rows (5.6 MB) and the
    1.6 MB FP64 output.  The row counts do not depend on the number of wavenumbers, so a
    narrow table on the same grids gives them."""
    import bench
    from oracle import oracle as O
    from paper_1912_07759_gb300 import synthetic as S
    tb = S.make_tables(2, 5, 22, 27, 64, with_cia=True)
    atm = S.config2_atmosphere()
    prof = O.profile(tb, atm)
    _, n_rows = method_bytes_from_profile(tb, prof["P"], prof["T"])
    n_cia = len({c + d for t in prof["T"] for c in [bracket_brute(tb.t_grid_cia, t)]
                 for d in (0, 1)})
    assert (n_rows, n_cia, len(tb.species)) == (65, 16, 7)
    W = 200000
    assert 5 * n_rows * W * 4 + 2 * n_cia * W * 4 + 7 * W * 4 + W * 8 == 292_800_000
    per_wn = bench.algorithmic_bytes(tb, atm) / tb.n_wn
    assert per_wn * W == 292_800_000


def test_roofline_fields_follow_their_definitions():
    """achieved = the method's bytes per launch / the mean launch time, frac = achieved / the
    measured peak, design_frac with the K write added, step_frac over the whole step; the FP32
    FMA peak of the FFMA contraction is SMs x 128 lanes x 2 FLOP x the SM clock passed in."""
    import bench
    from paper_1912_07759_gb300 import synthetic as S
    tb = S.make_tables(2, 5, 22, 27, 512, with_cia=True)
    atm = S.config2_atmosphere()
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0}
    total_ms, launches = 8.0, 100                          # 80 us per launch
    r = bench.roofline_of("k_opacity_fp32", (total_ms, launches), tb, atm, peaks, 2000.0, 148,
                          step_s=100e-6)
    alg = bench.algorithmic_bytes(tb, atm)
    assert r["algorithmic_bytes"] == alg and r["bound"] == "hbm" and r["peak"] == 6000.0
    assert abs(r["achieved"] - alg / 80e-6 / 1e9) < 0.1
    assert abs(r["frac"] - alg / 80e-6 / 1e9 / 6000.0) < 1e-4
    design = bench.algorithmic_bytes(tb, atm, "design_opacity")
    assert abs(r["design_frac"] - design / 80e-6 / 1e9 / 6000.0) < 1e-4
    assert abs(r["step_frac"] - alg / 100e-6 / 1e9 / 6000.0) < 1e-4
    f = bench.roofline_of("k_contract_fp32", (total_ms, launches), tb, atm, peaks, 2000.0, 148)
    N, W = atm.n_layers, tb.n_wn
    assert f["bound"] == "alu"
    assert abs(f["peak"] - 148 * 128 * 2 * 2000e6 / 1e12) < 0.1
    assert abs(f["achieved"] - 2.0 * W * N * (N + 1) / 2 / 80e-6 / 1e12) < 0.01
