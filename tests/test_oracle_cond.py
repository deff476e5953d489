"""Pins of the oracle's conservative conduction (div(K grad T) of Eq.
2675-eq1_Kath with harmonic-mean face conductances), each against something
other than the oracle: the centre form where K is uniform, exact energy
balance, the series-conduction steady state of a two-material slab, a dense
step matrix, and the adjoint against its transpose and finite differences."""
import numpy as np
import pytest

import oracle
import phantoms as ph
from tests import brute
from tests.test_oracle_adjoint import _loss_and_seed


def _hetero(case, k_tumor=1.6, k_vessel=0.3):
    case.table[ph.TUMOR].k = k_tumor
    case.table[ph.VESSEL].k = k_vessel
    return case


def test_uniform_K_equals_the_centre_form():
    case = ph.random_small_case(11, 12, 10, 9, power=5.0)
    for t in case.table:
        t.k = 0.52
    a = oracle.setup(case, "f64")
    b = oracle.setup(case, "f64", conduction="harmonic")
    sa, sb = oracle.initial_state(a), oracle.initial_state(b)
    oracle.run(a, sa, 80)
    oracle.run(b, sb, 80)
    assert np.allclose(sa.theta, sb.theta, rtol=0, atol=1e-12)


def test_energy_balance_with_heterogeneous_K():
    """No perfusion, insulated faces, no fixed voxels: the face fluxes cancel in
    pairs, so sum (rho c) h^3 theta = N dt P exactly; the centre form, whose
    fluxes are not antisymmetric where K changes, does not conserve it."""
    case = ph.random_small_case(12, 11, 10, 12, power=4.0, face_bc=ph.INSULATED, dt=0.05)
    lab = case.labels.copy()
    lab[lab == ph.VESSEL] = ph.TUMOR
    case.labels = lab
    for t in case.table:
        t.w_b = 0.0
    case.table[ph.TUMOR].k = 2.0
    case.table[ph.TUMOR].rho, case.table[ph.TUMOR].c = 1000.0, 3000.0
    N = 200
    res = {}
    for cond in ("harmonic", "centre"):
        m = oracle.setup(case, "f64", conduction=cond)
        st = oracle.initial_state(m)
        oracle.run(m, st, N)
        E = float(np.sum(m.rhoc * st.theta)) * case.h ** 3
        res[cond] = abs(E - N * case.dt * case.needle.power) / (N * case.dt * case.needle.power)
    assert res["harmonic"] < 1e-12
    assert res["centre"] > 1e-6


def test_two_material_slab_steady_state():
    """1-D slab, hot end held at theta0 and cold end at 0, K1 on the left and
    K2 on the right with the interface on a face: the steady flux F is the same
    through every face, F = theta0 / sum_f 1/K_f (the series resistance), and the
    profile is piecewise linear -- which is also the continuum solution at the
    voxel centres when the interface sits midway between two centres."""
    nx, h = 24, 1e-3
    K1, K2, th0 = 0.4, 1.6, 50.0
    labels = np.zeros((1, 1, nx), np.uint8)
    labels[..., nx // 2:] = 1
    labels[..., 0] = 2
    labels[..., -1] = 3
    t1, t2 = ph.Tissue(k=K1, w_b=0.0), ph.Tissue(k=K2, w_b=0.0)
    hot = ph.Tissue(k=K1, w_b=0.0, fixed=1, T_fixed_C=37.0 + th0)
    cold = ph.Tissue(k=K2, w_b=0.0, fixed=1, T_fixed_C=37.0)
    case = ph.Case("slab", nx, 1, 1, h, 0.2, 0, labels, [t1, t2, hot, cold],
                   ph.Needle(power=0.0), ph.Damage(enable=0), face_bc=ph.INSULATED)
    m = oracle.setup(case, "f64", conduction="harmonic")
    st = oracle.initial_state(m)
    oracle.run(m, st, 60000)
    Kvox = np.where(np.arange(nx) < nx // 2, K1, K2)
    Kf = 2 * Kvox[:-1] * Kvox[1:] / (Kvox[:-1] + Kvox[1:])
    F = th0 / np.sum(1.0 / Kf)
    expect = th0 - F * np.concatenate([[0.0], np.cumsum(1.0 / Kf)])
    assert np.allclose(st.theta[0, 0], expect, rtol=0, atol=1e-8)
    # continuum: linear in each material, flux continuity at the interface
    x = np.arange(nx) * h
    xi = (nx // 2 - 0.5) * h
    q = th0 / ((xi - 0) / K1 + (x[-1] - xi) / K2)
    cont = np.where(x < xi, th0 - q * x / K1, th0 - q * xi / K1 - q * (x - xi) / K2)
    assert np.allclose(st.theta[0, 0], cont, rtol=0, atol=1e-8)


@pytest.mark.parametrize("face_bc", [ph.DIRICHLET, ph.INSULATED])
def test_dense_step_matrix(face_bc):
    case = _hetero(ph.random_small_case(13, 8, 8, 8, face_bc=face_bc, power=3.0))
    m = oracle.setup(case, "bf16", conduction="harmonic")
    A, c = brute.step_matrix_faces(m.wf, m.b, m.s + m.qm, m.isfixed)
    N = 25
    st = oracle.initial_state(m)
    oracle.run(m, st, N)
    ref = brute.evolve(A, c, m.theta0.ravel(), N)
    assert np.allclose(st.theta.ravel(), ref, rtol=1e-12, atol=1e-12)


def test_adjoint_matches_dense_transpose():
    case = _hetero(ph.random_small_case(14, 6, 5, 7, nsteps=0, power=2.0))
    m = oracle.setup(case, "bf16", conduction="harmonic")
    A, _ = brute.step_matrix_faces(m.wf, m.b, m.s + m.qm, m.isfixed)
    rng = np.random.default_rng(1)
    lamN = rng.normal(size=m.a.shape)
    N = 29
    lam0, Lam, *_ = oracle.adjoint(m, N, lamN)
    v = lamN.ravel().copy()
    acc = np.zeros_like(v)
    for _ in range(N):
        acc += v
        v = A.T @ v
    assert np.allclose(lam0.ravel(), v, rtol=1e-12, atol=1e-14)
    assert np.allclose(Lam.ravel(), acc, rtol=1e-12, atol=1e-14)


def test_adjoint_gradients_match_central_fd():
    def mk():
        return _hetero(ph.random_small_case(21, 10, 9, 11, nsteps=0, power=6.0, h=1e-3, dt=0.1))
    case = mk()
    N = 60
    m = oracle.setup(case, "f64", conduction="harmonic")
    st = oracle.initial_state(m)
    oracle.run(m, st, N)
    rng = np.random.default_rng(3)
    sel = rng.random(m.a.shape) < 0.1
    target = st.theta + case.T_a_C + rng.normal(0, 2.0, size=m.a.shape)
    _, seed = _loss_and_seed(st.theta, case.T_a_C, target, sel)
    _, _, gk, gw, gP, gtip = oracle.adjoint(m, N, seed)

    def loss(c):
        mm = oracle.setup(c, "f64", conduction="harmonic")
        s2 = oracle.initial_state(mm)
        oracle.run(mm, s2, N)
        return _loss_and_seed(s2.theta, c.T_a_C, target, sel)[0]

    def fd(attr, l):
        x0 = getattr(case.table[l], attr)
        eps = 1e-4 * abs(x0)
        vals = []
        for sgn in (1, -1):
            c = mk()
            setattr(c.table[l], attr, x0 + sgn * eps)
            vals.append(loss(c))
        return (vals[0] - vals[1]) / (2 * eps)

    for l in (ph.LIVER, ph.TUMOR, ph.VESSEL):   # the vessel's K sets its face conductances
        assert gk[l] == pytest.approx(fd("k", l), rel=1e-5)
    for l in (ph.LIVER, ph.TUMOR):
        assert gw[l] == pytest.approx(fd("w_b", l), rel=1e-5)
    assert gk[ph.VESSEL] != 0.0 and gw[ph.VESSEL] == 0.0
