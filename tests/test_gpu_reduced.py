"""The reduced model of Sec. II (Eq. 8) on the GPU against the FP64 oracle
(oracle/reduced.py): the same Dormand-Prince steps in double precision, so
trajectories agree to round-off (the Bessel functions differ in their last
bits) over hundreds of steps, for one electron and a ragged number."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
from oracle import reduced as R

pytestmark = pytest.mark.gpu

PAR = dict(a0=2.0, omega_p=1 / 12.0, k_perp=0.04, v_phi=1.0008)


def _electrons(n, seed=5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-3.0, 3.0, n)
    zeta = rng.uniform(-40.0, -5.0, n)
    ux = rng.normal(0.0, 1.0, n)
    uz = rng.uniform(0.0, 60.0, n)
    return x, zeta, ux, uz


@pytest.mark.parametrize("n", [1, 1000])
def test_reduced_model_matches_oracle(n):
    y0 = _electrons(n)
    t0, dt, steps = 3.0, 0.05, 800
    g = q.reduced_integrate(*y0, PAR["a0"], PAR["omega_p"], PAR["k_perp"], PAR["v_phi"], t0, dt, steps)
    r = R.integrate(*y0, PAR["a0"], PAR["omega_p"], PAR["k_perp"], PAR["v_phi"], t0, dt, steps)
    for gk, rk in zip(g, r):
        assert np.max(np.abs(gk - rk) / (1.0 + np.abs(rk))) < 1e-8
    assert np.max(np.abs(g[2] - y0[2])) > 0.02               # the fields acted


def test_device_entry_point_and_edge_cases():
    import torch
    n = 300
    y0 = _electrons(n, seed=9)
    t0, dt, steps = 0.0, 0.1, 200
    host = q.reduced_integrate(*y0, PAR["a0"], PAR["omega_p"], PAR["k_perp"], PAR["v_phi"], t0, dt, steps)
    dev = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in y0]
    q.reduced_integrate_device([d.data_ptr() for d in dev], n, PAR["a0"], PAR["omega_p"], PAR["k_perp"],
                               PAR["v_phi"], t0, dt, steps)
    torch.cuda.synchronize()
    for h, d in zip(host, dev):
        assert np.array_equal(h, d.cpu().numpy())             # the same kernel: bit-identical
    same = q.reduced_integrate(*y0, PAR["a0"], PAR["omega_p"], PAR["k_perp"], PAR["v_phi"], t0, dt, 0)
    for s, v in zip(same, y0):
        assert np.array_equal(s, v)                            # zero steps leave the state
    empty = q.reduced_integrate([], [], [], [], PAR["a0"], PAR["omega_p"], PAR["k_perp"], PAR["v_phi"],
                                t0, dt, steps)
    assert all(len(v) == 0 for v in empty)
    with pytest.raises(q.QpicError):
        q.reduced_integrate(*y0, PAR["a0"], PAR["omega_p"], PAR["k_perp"], -1.0, t0, dt, steps)


def test_appendix_bunch_with_staggering_and_injection_matches_oracle():
    """Appendix A's injected bunch and parameters (a0 2.8, v_phi 1.002565,
    k_z 12.14 w_p, R 3 c/w_p), the regime the benchmark times, with the Yee
    staggering factor on the magnetic terms and injection spread over the
    first 200 steps: GPU and oracle agree to 1e-8"""
    import synth
    P = synth.REDUCED_PAPER
    wp = 1.0 / (P["v_phi"] * P["kz_over_wp"])
    kperp = 2.4 * wp / (P["R_over_lp"] + 1.0)
    n = 300
    y0 = synth.reduced_bunch(21, n, v_g=P["v_g"], wp=wp, R_over_lp=P["R_over_lp"])
    start = np.random.default_rng(4).integers(0, 200, n).astype(np.int32)
    start[:3] = (0, 399, 1000)                    # from the first step, on the last, never
    t0, dt, steps = 0.0, 0.05, 400
    for bfac in (1.0, np.cos(0.5 * 12.17 * 0.01875)):
        g = q.reduced_integrate(*y0, P["a0"], wp, kperp, P["v_phi"], t0, dt, steps, bfac=bfac, start=start)
        r = R.integrate(*y0, P["a0"], wp, kperp, P["v_phi"], t0, dt, steps, bfac=bfac, start=start)
        for gk, rk in zip(g, r):
            assert np.max(np.abs(gk - rk) / (1.0 + np.abs(rk))) < 1e-8, bfac
        assert all(gk[2] == yk[2] for gk, yk in zip(g, y0))        # never injected: unchanged
        assert np.max(np.abs(g[2][:2] - y0[2][:2])) > 0             # the others moved
