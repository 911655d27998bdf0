"""Work partition pins (Sec. III.B): the directional work of Eq. 17 (track
mode 2: W0 = W_z, W1 = W_perp) next to the modal work of Eq. 16 (mode 1), and
the f-corrected estimate of Eqs. 19-20 in the oracle and in the library's host
function.

- the two splits share one total: W_z + W_perp = W_LWFA + W_DLA per particle
  (both are q dt E.v summed two ways), on an evolving laser-plasma box;
- one electron in a uniform longitudinal field (m = 0 E_z): W_perp = 0 and
  W_z = W_LWFA = gamma - 1 (work-energy theorem, to the push's O(dt^2));
- one electron in a uniform transverse field (m = 1 E_x): W_z = 0 and
  W_perp = W_DLA = gamma - 1;
- Eq. 19's f against the cycle-averaged works of the focused laser fields of
  Eq. 18 along a resonant betatron orbit, by quadrature;
- the library's qpic_work_f_estimate against the oracle's, the total of the
  two estimates, and its argument checks (host code, no GPU).
"""
import numpy as np
import pytest

from oracle import coeffs as C
from oracle import diag, setup

DZ, DR, DT = 0.2, 0.5, 0.12


def _box(oracle_mod, mode, nz=32, nr=16):
    cE, cB = C.dual_coefficients(DT, DZ)
    return oracle_mod.Oracle(nz, nr, 2, DZ, DR, DT, cE, cB, C.filter_taps(cB), periodic=True,
                             track_work=mode)


def _one_electron(o, r=0.6, phi=0.3):
    one = np.ones(1)
    o.load_particles(3.2 * one, r * one, phi * one, 0 * one, 0 * one, 0 * one, 1e-12 * one)


def test_directional_and_modal_work_share_the_total(oracle_mod):
    """a laser (a0 = 2) in a plasma, 12 steps, once per mode from the same state"""
    res = {}
    for mode in (1, 2):
        o = _box(oracle_mod, mode, nz=96, nr=20)
        cE, cB = C.dual_coefficients(DT, DZ)
        parts = setup.plasma_cells(np.arange(96), 20, DZ, DR, 0.01, 0.0, 0.0, (2, 2, 2), 11)
        o.load_particles(**parts)
        setup.add_laser(o, cE, cB, 2.0, 6.0, 8.0, 9.6, 9.6)
        o.step(12)
        res[mode] = o.particles()
    a, b = res[1], res[2]
    for k in ("z", "r", "ux", "uy", "uz"):                 # same trajectories
        assert np.array_equal(a[k], b[k]), k
    tot_modal, tot_dir = a["W0"] + a["W1"], b["W0"] + b["W1"]
    scale = np.abs(tot_modal).max()
    assert scale > 1e-4
    assert np.max(np.abs(tot_modal - tot_dir)) <= 1e-12 * scale
    # the laser's longitudinal field does work too: W_z is not the modal m = 0 work
    assert np.max(np.abs(b["W0"] - a["W0"])) > 1e-3 * scale


@pytest.mark.parametrize("mode", [1, 2])
def test_uniform_longitudinal_field(oracle_mod, mode):
    o = _box(oracle_mod, mode)
    E0 = 0.02
    o.set_field("E", "z", 0, np.full((o.nr + 1, o.nz), E0, dtype=complex))
    _one_electron(o)
    o.step(20)
    p = o.particles()
    gamma = np.sqrt(1 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)[0]
    assert p["uz"][0] < 0                                   # q = -1: pushed towards -z
    # mode 1: W0 = W_LWFA (m = 0), W1 = W_DLA; mode 2: W0 = W_z, W1 = W_perp
    assert abs(p["W1"][0]) <= 1e-9 * (gamma - 1)
    assert p["W0"][0] > 0
    assert abs(p["W0"][0] - (gamma - 1)) <= 1e-4 * (gamma - 1)


@pytest.mark.parametrize("mode", [1, 2])
def test_uniform_transverse_field(oracle_mod, mode):
    """E_x = E0 everywhere: the m = 1 parts E_r^1 = E0/2, E_phi^1 = i E0/2"""
    o = _box(oracle_mod, mode)
    E0 = 0.02
    shape = (o.nr + 1, o.nz)
    o.set_field("E", "r", 1, np.full(shape, 0.5 * E0, dtype=complex))
    o.set_field("E", "phi", 1, np.full(shape, 0.5j * E0))
    _one_electron(o)
    o.step(20)
    p = o.particles()
    gamma = np.sqrt(1 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)[0]
    assert p["ux"][0] < 0 and abs(p["uy"][0]) < 1e-9 * abs(p["ux"][0])
    # mode 1: W0 = W_LWFA = 0 (no m = 0 field); mode 2: W0 = W_z = 0 (no E_z)
    assert abs(p["W0"][0]) <= 1e-9 * (gamma - 1)
    assert p["W1"][0] > 0
    assert abs(p["W1"][0] - (gamma - 1)) <= 1e-4 * (gamma - 1)


@pytest.mark.parametrize("gamma,omega_p,w0", [(100.0, 0.1, 10.0), (400.0, 1 / 12.0, 2.53 * 12.0)])
def test_f_ratio_from_the_laser_fields(gamma, omega_p, w0):
    """Eq. 19 from Eq. 18: x = A cos(w_b t), theta = w_b t, v_z = c = 1,
    k_z = omega0 = 1, A << w0; the works over one betatron period by quadrature"""
    wb = omega_p / np.sqrt(2 * gamma)
    A = 1e-3 * w0
    t = np.linspace(0.0, 2 * np.pi / wb, 200001)
    x, vx = A * np.cos(wb * t), -A * wb * np.sin(wb * t)
    env = np.exp(-x ** 2 / w0 ** 2)
    Ex = env * np.sin(wb * t)
    Ez = 2 * x / w0 ** 2 * env * np.cos(wb * t)
    Wz = -np.trapezoid(Ez * 1.0, t)
    Wperp = -np.trapezoid(Ex * vx, t)
    assert Wperp > 0                                      # in phase: the laser gives energy
    assert diag.work_f_ratio(gamma, omega_p, w0) == pytest.approx(Wz / Wperp, rel=1e-5)


def test_library_f_estimate_matches_the_oracle():
    import paper_2303_12874_gb300 as q
    rng = np.random.default_rng(19)
    n = 1000
    u = rng.normal(0, 30, (3, n))
    u[2] += 200
    Wz, Wp = rng.normal(100, 50, n), rng.normal(50, 30, n)
    lw, dl = q.work_f_estimate(u[0], u[1], u[2], Wz, Wp, 1 / 12.0, 30.36)
    gamma = np.sqrt(1 + (u ** 2).sum(0))
    rl, rd = diag.work_f_estimate(gamma, Wz, Wp, 1 / 12.0, 30.36)
    assert np.allclose(lw, rl, rtol=1e-13, atol=1e-12) and np.allclose(dl, rd, rtol=1e-13, atol=1e-12)
    assert np.allclose(lw + dl, Wz + Wp, rtol=1e-12)      # the estimate splits the same total
    assert np.all(diag.work_f_ratio(gamma, 1 / 12.0, 30.36) < 0)
    with pytest.raises(q.QpicError):
        q.work_f_estimate(u[0], u[1], u[2], Wz, Wp, 0.0, 30.36)
    L = q.load()
    assert L.qpic_work_f_estimate(-1, None, None, None, None, None, 0.1, 1.0, 1.0, None, None) == -1


def test_f_at_the_papers_bunch_values():
    """Sec. IV.C evaluates Eq. 19 with omega0 = 12 omega_p and w0 = 2.53 c/omega_p:
    in units of omega0, omega_p = 1/12 and w0 = 30.36, so f = -0.0260 sqrt(2 gamma)
    and f(gamma = 200) = -0.52"""
    f = diag.work_f_ratio(200.0, 1 / 12.0, 2.53 * 12.0)
    assert f == pytest.approx(-0.5208, abs=5e-4)
    assert diag.work_f_ratio(50.0, 1 / 12.0, 2.53 * 12.0) / np.sqrt(100.0) == pytest.approx(-0.02604, abs=5e-5)
