"""Pins of the oracle's discrete adjoint: dense transpose at small size and
central finite differences (eps = 1e-4 relative) of the FP64 forward."""
import math

import numpy as np
import pytest

import oracle
import phantoms as ph
from tests import brute


def _loss_and_seed(theta, T_a, target, sel, width=1.0, thr=60.0):
    """Final-temperature MSE on a voxel subset plus the smoothed necrosis
    volume fraction mean(sigmoid((T - thr)/width)); returns (L, dL/dtheta)."""
    T = theta + T_a
    d = T[sel] - target[sel]
    sig = 1.0 / (1.0 + np.exp(-(T - thr) / width))
    L = float(np.mean(d * d) + np.mean(sig))
    g = np.zeros_like(theta)
    g[sel] = 2.0 * d / d.size
    g += sig * (1 - sig) / width / theta.size
    return L, g


@pytest.mark.parametrize("face_bc", [ph.DIRICHLET, ph.INSULATED])
def test_adjoint_matches_dense_transpose(face_bc):
    # insulated faces give free voxels with fewer than six neighbours
    case = ph.random_small_case(5, 6, 5, 7, face_bc=face_bc, nsteps=0, power=2.0)
    m = oracle.setup(case, "bf16")
    A, _ = brute.step_matrix(m.a, m.b, m.s + m.qm, m.isfixed)
    rng = np.random.default_rng(0)
    lamN = rng.normal(size=m.a.shape)
    N = 37
    lam0, Lam, *_ = oracle.adjoint(m, N, lamN)
    AT = A.T
    v = lamN.ravel().copy()
    acc = np.zeros_like(v)
    for _ in range(N):
        acc += v
        v = AT @ v
    assert np.allclose(lam0.ravel(), v, rtol=1e-12, atol=1e-14)
    assert np.allclose(Lam.ravel(), acc, rtol=1e-12, atol=1e-14)


def _fd_setup():
    case = ph.random_small_case(21, 10, 9, 11, nsteps=0, power=6.0, h=1e-3, dt=0.1)
    return case


def _forward_loss(case, N, target, sel):
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    oracle.run(m, st, N)
    return _loss_and_seed(st.theta, case.T_a_C, target, sel)[0]


def test_adjoint_gradients_match_central_fd():
    case = _fd_setup()
    N = 60
    m = oracle.setup(case, "f64")
    st = oracle.initial_state(m)
    oracle.run(m, st, N)
    rng = np.random.default_rng(3)
    sel = rng.random(m.a.shape) < 0.1
    target = st.theta + case.T_a_C + rng.normal(0, 2.0, size=m.a.shape)
    L0, seed = _loss_and_seed(st.theta, case.T_a_C, target, sel)
    _, _, gk, gw, gP, gtip = oracle.adjoint(m, N, seed)

    def fd(mutate, x0):
        eps = 1e-4 * abs(x0)
        vals = []
        for sgn in (1, -1):
            c = _fd_setup()
            mutate(c, x0 + sgn * eps)
            vals.append(_forward_loss(c, N, target, sel))
        return (vals[0] - vals[1]) / (2 * eps)

    def set_k(l):
        def f(c, v):
            c.table[l].k = v
        return f

    def set_wb(l):
        def f(c, v):
            c.table[l].w_b = v
        return f

    for l in (ph.LIVER, ph.TUMOR):
        g_fd = fd(set_k(l), case.table[l].k)
        assert gk[l] == pytest.approx(g_fd, rel=1e-5)
        g_fd = fd(set_wb(l), case.table[l].w_b)
        assert gw[l] == pytest.approx(g_fd, rel=1e-5)
    # a fixed (vessel) label has no influence
    assert gk[ph.VESSEL] == 0.0 and gw[ph.VESSEL] == 0.0

    def set_P(c, v):
        c.needle.power = v
    assert gP == pytest.approx(fd(set_P, case.needle.power), rel=1e-5)

    # tip: no voxel centre may sit where the clamp kink d = r0 is crossed
    eps_tip = 1e-4 * max(abs(t) for t in case.needle.tip)
    assert np.min(np.abs(m.dist - case.needle.r_clamp)) > 3 * eps_tip
    for axis in range(3):
        def set_tip(c, v, axis=axis):
            tp = list(c.needle.tip)
            tp[axis] = v
            c.needle.tip = tuple(tp)
        x0 = case.needle.tip[axis]
        g_fd = fd(set_tip, x0)
        assert gtip[axis] == pytest.approx(g_fd, rel=1e-5, abs=1e-9 * np.max(np.abs(gtip)))
