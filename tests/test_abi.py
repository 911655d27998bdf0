"""The C ABI: the library builds for sm_103a, loads, exports every function
declared in include/qpic.h, and its host-only numerics (coefficient fit,
filter taps, stability limit) agree with the oracle's independent ones.
No GPU is needed; a context refuses to start without one (no CPU fallback)."""
import os
import re

import numpy as np
import pytest

import paper_2303_12874_gb300 as q
from oracle import coeffs as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qpic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qpic_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = q.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("nu", [0.4, 0.7, 0.85])
def test_host_fit_matches_oracle(nu):
    dz = 0.2
    cE, cB = q.fit_coefficients("dual", nu * dz, dz)
    oE, oB = C.dual_coefficients(nu * dz, dz)
    assert np.max(np.abs(cE - oE)) < 1e-11
    assert np.max(np.abs(cB - oB)) < 1e-11
    yE, yB = q.fit_coefficients("yee", nu * dz, dz)
    assert list(yE) == [1.0] and list(yB) == [1.0]


def test_host_filter_taps_match_oracle():
    _, cB = C.dual_coefficients(0.14, 0.2)
    k_lib = q.filter_taps(cB)
    k_or = C.filter_taps(cB)
    n = min(len(k_lib), len(k_or))
    assert abs(len(k_lib) - len(k_or)) <= 1        # the 1e-16 cut may fall either side
    assert np.max(np.abs(k_lib[:n] - k_or[:n])) < 1e-13
    assert q.filter_taps(np.array([1.0])) is None


@pytest.mark.parametrize("solver", ["dual", "yee"])
def test_host_stability_limit_matches_oracle(solver):
    lib = q.stability_limit(solver, 0.2, 0.5, 32, 2)
    ora = C.cfl_dt(0.2, 0.5, 32, 2, solver)
    assert abs(lib / ora - 1) < 1e-8


def test_context_needs_a_gpu():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(q.QpicError):
        q.Sim(64, 8, 0.2, 0.5)


def test_reduced_model_argument_checks_without_a_gpu():
    """qpic_reduced_integrate refuses bad arguments before touching the GPU,
    accepts an empty set, and reports a CUDA error (no CPU fallback) otherwise
    when no GPU is present"""
    import math
    L = q.load()
    ok = (1.0, 0.1, 0.04, 1.0, 1.0, 0.0, 0.1, 1, None)     # a0, w_p, k_perp, v_phi, bfac, t0, dt, nsteps, start
    assert L.qpic_reduced_integrate(0, None, None, None, None, *ok) == 0
    assert L.qpic_reduced_integrate(-1, None, None, None, None, *ok) == -1
    for k, bad in ((3, -1.0), (3, 0.0), (5, math.nan), (6, 0.0), (6, math.inf), (2, -0.1), (7, -1),
                   (4, math.inf)):
        args = list(ok)
        args[k] = bad
        assert L.qpic_reduced_integrate(0, None, None, None, None, *args) == -1, (k, bad)
    x = np.zeros(3)
    assert L.qpic_reduced_integrate(3, q._dp(x), None, q._dp(x), q._dp(x), *ok) == -1
    import torch
    if not torch.cuda.is_available():
        y = [np.zeros(2) for _ in range(4)]
        assert L.qpic_reduced_integrate(2, *[q._dp(v) for v in y], *ok) != 0


def test_configuration_checks_come_before_the_gpu():
    """qpic_init validates its configuration before it touches the device: an
    unknown work-tracking mode or precision is named in the error (with or
    without a GPU)"""
    with pytest.raises(q.QpicError, match="track_work"):
        q.Sim(64, 8, 0.2, 0.5, track_work=3)
    with pytest.raises(q.QpicError, match="precision"):
        q.Sim(64, 8, 0.2, 0.5, precision=7)
