"""The seeded input recipe against the workloads it stands in for: grid extents, table value
ranges, the two fixed atmospheres, the prior ranges of the batched draws, the bins and the
observation noise.  These pins keep the synthetic inputs shaped like the paper's workloads
(Sec. 8: 100 layers from 1e6 to 1e-4 Pa, H2/He background, cross-sections of order 1e-22 cm^2
with line structure, a retrieval over 1.1-1.7 micron at R ~ 100)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1912_07759_gb300 import synthetic as S  # noqa: E402


def test_table_grids_and_values():
    tb = S.make_tables(1, 2, 13, 15, 4000, with_cia=True)
    assert tb.sigma.shape == (2, 13, 15, 4000) and tb.sigma.dtype == np.float32
    assert np.isclose(tb.t_grid[0], 300.0) and np.isclose(tb.t_grid[-1], 3000.0)
    assert np.isclose(tb.wn_grid[0], 300.0) and np.isclose(tb.wn_grid[-1], 30000.0)
    # log-uniform native grid: constant resolution
    r = tb.wn_grid[1:] / tb.wn_grid[:-1]
    assert np.allclose(r, r[0], rtol=1e-9)
    assert np.all(np.diff(np.log(tb.p_grid)) > 0)
    # sigma in m^2: the cm^2 log10 values lie in [-33, -17], the continuum near -22
    lg_cm2 = np.log10(tb.sigma.astype(np.float64)) + 4.0
    assert lg_cm2.min() >= -33.0 - 1e-4 and lg_cm2.max() <= -17.0 + 1e-4
    assert abs(np.median(lg_cm2) - (-22.0)) < 1.5
    # line spikes: the upper tail sits well above the median at every (P, T)
    q = np.percentile(lg_cm2, [50, 99.5], axis=-1)
    assert np.all(q[1] - q[0] > 0.5)
    # fill gases H2 and He after the absorbers; CIA pairs H2-H2 and H2-He
    assert tb.species[-2:] == ("H2", "He")
    assert [tuple(p) for p in tb.cia_pair] == [(2, 2), (2, 3)]
    # seeded: the same call gives the same tables
    tb2 = S.make_tables(1, 2, 13, 15, 4000, with_cia=True)
    assert np.array_equal(tb.sigma, tb2.sigma)


def test_fixed_atmospheres():
    a1 = S.config1_atmosphere()
    assert (a1.n_layers, a1.p_max, a1.p_min) == (100, 1e6, 1e-4)
    assert list(a1.tnode_t) == [1500.0]
    assert np.allclose(10.0 ** a1.log10_x, [1e-4, 1e-5])
    assert np.allclose(a1.fill_frac, [0.83, 0.17])
    a2 = S.config2_atmosphere()
    assert a2.n_layers == 100 and a2.log10_x.shape == (5,)
    assert np.all((a2.log10_x >= -8.0) & (a2.log10_x <= -3.0))
    assert a2.tnode_t.shape == (4,) and a2.tnode_t.min() >= 800.0 and a2.tnode_t.max() <= 2200.0
    assert a2.p_cloud_top == 1e3


def test_prior_draws_and_layer_counts():
    spec = S.batch_spec(5)
    th = S.draw_theta(7, 4096, spec)
    assert th.shape == (4096, spec.n_theta) == (4096, 5 + 4 + 2)
    lx, t, rp, lpc = th[:, :5], th[:, 5:9], th[:, 9], th[:, 10]
    assert lx.min() >= -12.0 and lx.max() <= -1.0
    assert t.min() >= 500.0 and t.max() <= 2500.0
    assert rp.min() >= 0.8 and rp.max() <= 1.5
    assert lpc.min() >= 2.0 and lpc.max() <= 6.0          # cloud top 1e2 - 1e6 Pa
    # uniform priors: the draws cover their ranges
    assert lx.min() < -11.9 and lx.max() > -1.1 and t.min() < 510.0 and t.max() > 2490.0
    nl = S.draw_nlayers(8, 4096)
    assert nl.min() == 50 and nl.max() == 150 and nl.dtype == np.int32


def test_bins_and_noise():
    c, w = S.bins_logspaced()
    assert c.shape == w.shape == (50,)
    assert np.isclose(c[0] - w[0] / 2, 1.1) and np.isclose(c[-1] + w[-1] / 2, 1.7)
    R = c / w
    assert 100.0 <= R.min() and R.max() <= 130.0            # R ~ 100 over 1.1-1.7 micron
    sig, z = S.obs_noise(3, 50)
    assert sig.min() >= 30e-6 and sig.max() <= 100e-6 and z.shape == (50,)
