"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the oracle function it pins and the fact it uses.  Nothing
here re-types an oracle formula and compares it with itself: the checks are
values printed by the paper, kernel identities that define the published
delta kernels, closed forms of Algorithm 1, conservation laws, and a dense
brute force that evaluates every (marker, cell) pair over periodic images.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2408_14140_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pvf_tables.txt")
KERNELS = [oracle.ROMA3, oracle.PESKIN4]
SUPPORT = {oracle.ROMA3: 1.5, oracle.PESKIN4: 2.0}
SUM_SQ = {oracle.ROMA3: 0.5, oracle.PESKIN4: 0.375}


# ---------------------------------------------------------------- delta kernel
@pytest.mark.parametrize("kernel", KERNELS)
def test_phi_moment_conditions(kernel):
    """or_phi: partition of unity, zero first moment and constant sum of
    squares at every offset -- the conditions that define the Roma-Peskin-
    Berger three-point kernel and Peskin's four-point kernel."""
    rng = np.random.default_rng(1)
    for r in np.concatenate([rng.uniform(0, 1, 200), [0.0, 0.25, 0.5, 0.75]]):
        js = np.arange(-3, 5)
        w = np.array([oracle.phi(kernel, r - j) for j in js])
        assert abs(w.sum() - 1.0) < 4e-16
        assert abs(np.sum((r - js) * w)) < 4e-16
        assert abs(np.sum(w * w) - SUM_SQ[kernel]) < 4e-16
        if kernel == oracle.PESKIN4:
            even = sum(oracle.phi(kernel, r - j) for j in js if j % 2 == 0)
            assert abs(even - 0.5) < 4e-16


@pytest.mark.parametrize("kernel", KERNELS)
def test_phi_support_and_symmetry(kernel):
    """or_phi: even, non-negative, zero outside its support, continuous at the
    piece boundaries."""
    S = SUPPORT[kernel]
    for r in np.linspace(0, S + 1, 401):
        v = oracle.phi(kernel, r)
        assert v == oracle.phi(kernel, -r)
        assert v >= 0.0
        if r >= S:
            assert v == 0.0
    for b in ([0.5, 1.5] if kernel == oracle.ROMA3 else [1.0, 2.0]):
        assert abs(oracle.phi(kernel, b - 1e-12) - oracle.phi(kernel, b + 1e-12)) < 1e-10


# ------------------------------------------------------------------ helpers
def dense_W(n, h, org, X, kernel):
    """Brute-force interpolation matrix W[M, N]: for every marker and every
    cell, the product of 1-D kernel values summed over the periodic images of
    the marker (no stencil bookkeeping)."""
    n = list(n)
    M = X.shape[0]
    W = np.zeros((M,) + (n[2], n[1], n[0]))
    for l in range(M):
        ax = []
        for a in range(3):
            s = (X[l, a] - org[a]) / h - 0.5
            wa = np.zeros(n[a])
            for c in range(n[a]):
                for img in range(-2, 3):
                    wa[c] += oracle.phi(kernel, s - c - img * n[a])
            ax.append(wa)
        W[l] = ax[2][:, None, None] * ax[1][None, :, None] * ax[0][None, None, :]
    return W.reshape(M, -1)


def tiny_grid(seed, n=(6, 7, 8)):
    rng = np.random.default_rng(seed)
    h = 0.1
    org = rng.uniform(-1, 1, 3)
    u = rng.normal(size=(3, n[2], n[1], n[0]))
    return n, h, org, u, rng


# ------------------------------------------------------------- interpolation
@pytest.mark.parametrize("kernel", KERNELS)
def test_interpolate_matches_dense_brute_force(kernel):
    """or_interpolate == W u with W from every cell and periodic image,
    markers anywhere (including across the periodic seam)."""
    n, h, org, u, rng = tiny_grid(2)
    X = org + rng.uniform(-0.5, 1.5, (13, 3)) * np.array(n) * h
    W = dense_W(n, h, org, X, kernel)
    U = oracle.interpolate(n, h, org, u, X, kernel)
    ref = np.stack([W @ u[c].ravel() for c in range(3)], axis=1)
    assert np.max(np.abs(U - ref)) < 1e-13


@pytest.mark.parametrize("kernel", KERNELS)
def test_interpolate_exact_for_linear_fields(kernel):
    """or_interpolate reproduces u = a + B x exactly away from the seam (a
    consequence of the kernel's zeroth and first moment conditions)."""
    n = (32, 32, 32)
    h = 1.0 / 32
    org = np.zeros(3)
    rng = np.random.default_rng(3)
    a = rng.normal(size=3)
    B = rng.normal(size=(3, 3))
    xs = (np.arange(32) + 0.5) * h
    Z, Y, Xg = np.meshgrid(xs, xs, xs, indexing="ij")
    u = np.stack([a[c] + B[c, 0] * Xg + B[c, 1] * Y + B[c, 2] * Z for c in range(3)])
    X = rng.uniform(0.3, 0.7, (50, 3))
    U = oracle.interpolate(n, h, org, u, X, kernel)
    assert np.max(np.abs(U - (a + X @ B.T))) < 1e-13


# ------------------------------------------------------------------ spreading
@pytest.mark.parametrize("kernel", KERNELS)
def test_spread_matches_dense_brute_force(kernel):
    """or_spread == W^T (F dV) / h^3, and it accumulates into f."""
    n, h, org, _, rng = tiny_grid(4)
    X = org + rng.uniform(-0.5, 1.5, (11, 3)) * np.array(n) * h
    F = rng.normal(size=(11, 3))
    dV = rng.uniform(0.5, 2.0, 11) * h ** 3
    W = dense_W(n, h, org, X, kernel)
    f0 = rng.normal(size=(3, n[2], n[1], n[0]))
    f = oracle.spread(n, h, org, X, F, dV, kernel, f=f0.copy())
    ref = f0 + np.stack([(W.T @ (F[:, c] * dV)).reshape(n[2], n[1], n[0])
                         for c in range(3)]) / h ** 3
    assert np.max(np.abs(f - ref)) < 1e-12


@pytest.mark.parametrize("kernel", KERNELS)
def test_spread_conserves_force_and_torque(kernel):
    """Sum_c f_c h^3 = sum_l F_l dV_l and sum_c (x_c - X0) x f_c h^3 =
    sum_l (X_l - X0) x F_l dV_l (Sec. 1: kernels conserving total force and
    torque on uniform grids)."""
    n = (24, 24, 24)
    h = 1.0 / 24
    org = np.zeros(3)
    rng = np.random.default_rng(5)
    X = rng.uniform(0.3, 0.7, (40, 3))
    F = rng.normal(size=(40, 3))
    dV = rng.uniform(0.5, 1.5, 40) * h ** 3
    f = oracle.spread(n, h, org, X, F, dV, kernel)
    tot = f.reshape(3, -1).sum(axis=1) * h ** 3
    assert np.allclose(tot, (F * dV[:, None]).sum(axis=0), atol=1e-14, rtol=0)
    xs = (np.arange(24) + 0.5) * h
    Z, Y, Xg = np.meshgrid(xs, xs, xs, indexing="ij")
    x0 = np.array([0.5, 0.5, 0.5])
    r = np.stack([Xg - x0[0], Y - x0[1], Z - x0[2]])
    torque_f = np.cross(r.reshape(3, -1).T, f.reshape(3, -1).T).sum(axis=0) * h ** 3
    torque_m = np.cross(X - x0, F * dV[:, None]).sum(axis=0)
    assert np.allclose(torque_f, torque_m, atol=1e-14, rtol=0)


@pytest.mark.parametrize("kernel", KERNELS)
def test_spread_interpolate_adjoint(kernel):
    """sum_l dV_l F_l . (J u)_l = h^3 sum_c u_c . (S F)_c (Sec. 2: S and J
    adjoint), markers anywhere including across the seam."""
    n, h, org, u, rng = tiny_grid(6, n=(9, 8, 10))
    X = org + rng.uniform(-1, 2, (30, 3)) * np.array(n) * h
    F = rng.normal(size=(30, 3))
    dV = rng.uniform(0.5, 1.5, 30) * h ** 3
    lhs = np.sum(dV[:, None] * F * oracle.interpolate(n, h, org, u, X, kernel))
    rhs = h ** 3 * np.sum(u * oracle.spread(n, h, org, X, F, dV, kernel))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


# --------------------------------------------------------------- Algorithm 1
def _one_particle(X0, R, dV, U, W):
    return (np.asarray(X0, float).reshape(1, 3), np.asarray(U, float).reshape(1, 3),
            np.asarray(W, float).reshape(1, 3), np.array([0, R.shape[0]]), R, dV)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("Ns", [1, 2, 3, 5])
def test_multidirect_single_marker_closed_form(kernel, Ns):
    """Algorithm 1 with one isolated marker: the slip error contracts as
    e^m = (1 - kappa)^m e^0 with kappa = (dV/h^3) (sum phi^2)^3, for any
    marker position; and F^Ns = e^0 (1 - (1-kappa)^Ns) / (kappa dt)."""
    n = (16, 16, 16)
    h = 1.0 / 16
    org = np.zeros(3)
    rng = np.random.default_rng(7 + Ns)
    u = rng.normal(size=(3, 16, 16, 16))
    Xr = rng.uniform(0.2, 0.8, 3)
    R = rng.uniform(-0.05, 0.05, (1, 3))
    dV = np.array([0.8 * h ** 3])
    Ur, Wr = rng.normal(size=3), rng.normal(size=3)
    dt = 3e-3
    Ud = Ur + np.cross(Wr, R[0])
    e0 = Ud - oracle.interpolate(n, h, org, u, Xr + R, kernel)[0]
    un, F, _ = oracle.multidirect(n, h, org, u, *_one_particle(Xr, R, dV, Ur, Wr),
                                  Ns, dt, kernel)
    eN = Ud - oracle.interpolate(n, h, org, un, Xr + R, kernel)[0]
    kap = 0.8 * SUM_SQ[kernel] ** 3
    assert np.allclose(eN, (1 - kap) ** Ns * e0, atol=1e-12, rtol=0)
    assert np.allclose(F[0] * dt, e0 * (1 - (1 - kap) ** Ns) / kap, atol=1e-12, rtol=0)


def _dense_alg1(W, u0, Ud, dV, h, Ns, dt):
    """Algorithm 1 in dense linear algebra, cumulative form."""
    F = np.zeros_like(Ud)
    u = u0.copy()
    for _ in range(Ns):
        U = np.stack([W @ u[c] for c in range(3)], axis=1)
        F = F + (Ud - U) / dt
        f = np.stack([W.T @ (F[:, c] * dV) for c in range(3)]) / h ** 3
        u = u0 + dt * f
    return u, F, f


@pytest.mark.parametrize("kernel", KERNELS)
def test_multidirect_multi_marker_dense(kernel):
    """Several coupled markers on a tiny periodic grid: the slip error obeys
    e^m = (I - K)^m e^0 with K_lk = (dV_k/h^3) sum_c w_lc w_kc, and u, F, f
    match a dense evaluation of Algorithm 1."""
    n, h, org, u, rng = tiny_grid(8, n=(8, 8, 8))
    M = 12
    Xr = org + 0.5 * np.array(n) * h
    R = rng.uniform(-0.25, 0.25, (M, 3))
    dV = rng.uniform(0.5, 1.2, M) * h ** 3
    Ur, Wr = rng.normal(size=3), rng.normal(size=3)
    Ns, dt = 3, 2e-3
    X = Xr + R
    Ud = Ur + np.cross(Wr, R)
    W = dense_W(n, h, org, X, kernel)
    uf = u.reshape(3, -1)
    un, F, f = oracle.multidirect(n, h, org, u, *_one_particle(Xr, R, dV, Ur, Wr),
                                  Ns, dt, kernel, want_f=True)
    ud, Fd, fd = _dense_alg1(W, uf, Ud, dV, h, Ns, dt)
    scale = np.max(np.abs(ud))
    assert np.max(np.abs(un.reshape(3, -1) - ud)) < 1e-12 * scale
    assert np.max(np.abs(F - Fd)) < 1e-12 * np.max(np.abs(Fd))
    assert np.max(np.abs(f.reshape(3, -1) - fd)) < 1e-12 * np.max(np.abs(fd))
    K = (W @ W.T) * dV[None, :] / h ** 3
    e0 = Ud - np.stack([W @ uf[c] for c in range(3)], axis=1)
    eN = Ud - np.stack([W @ un.reshape(3, -1)[c] for c in range(3)], axis=1)
    pred = np.linalg.matrix_power(np.eye(M) - K, Ns) @ e0
    assert np.max(np.abs(eN - pred)) < 1e-11 * np.max(np.abs(e0))


@pytest.mark.parametrize("order", [oracle.SEQUENTIAL, oracle.SIMULTANEOUS])
def test_multidirect_dt_invariance(order):
    """u(Ns) does not depend on dt and F scales as 1/dt (dt cancels between
    the force update and the velocity correction of Algorithm 1)."""
    case = synth.cluster_case(N=48, P=3, D_cells=8, phi=0.15, K=4, Ns=3, seed=3)
    args = (case.n, case.h, case.org, case.u, case.Xr, case.Ur, case.Wr,
            case.moff, case.R, case.dV, 3)
    u1, F1, _ = oracle.multidirect(*args, 1e-3, order=order)
    u2, F2, _ = oracle.multidirect(*args, 7e-2, order=order)
    assert np.max(np.abs(u1 - u2)) < 1e-12 * np.max(np.abs(u1))
    assert np.max(np.abs(F1 * 1e-3 - F2 * 7e-2)) < 1e-12 * np.max(np.abs(F1 * 1e-3))


def test_multidirect_orders_agree_for_disjoint_bands():
    """Sequential and simultaneous particle orders coincide when no two
    particles' kernel supports overlap, and differ when they do."""
    N = 64
    h = 1.0 / N
    rng = synth.SplitMix64(11)
    u = synth.fourier_field((N, N, N), 6, rng, h)
    Rm, dv = synth.sphere_markers(5 * h, h)
    M1 = Rm.shape[0]
    Ur = 0.1 * rng.normals(6).reshape(2, 3)
    Wr = 0.1 * rng.normals(6).reshape(2, 3)
    moff = [0, M1, 2 * M1]
    R = np.concatenate([Rm, Rm])
    dV = np.concatenate([dv, dv])
    far = np.array([[0.25, 0.3, 0.3], [0.75, 0.6, 0.7]])
    near = np.array([[0.4, 0.5, 0.5], [0.4 + 12 * h, 0.5, 0.5]])
    for Xr, same in ((far, True), (near, False)):
        a = oracle.multidirect((N,) * 3, h, (0, 0, 0), u, Xr, Ur, Wr, moff, R, dV, 3,
                               1e-3, order=oracle.SEQUENTIAL)
        b = oracle.multidirect((N,) * 3, h, (0, 0, 0), u, Xr, Ur, Wr, moff, R, dV, 3,
                               1e-3, order=oracle.SIMULTANEOUS)
        d = np.max(np.abs(a[0] - b[0]))
        if same:
            assert d == 0.0 and np.array_equal(a[1], b[1])
        else:
            assert d > 1e-6


def test_multidirect_sequential_matches_dense_chain():
    """Sequential order with two overlapping particles == Algorithm 1 run in
    dense algebra for particle 0, then for particle 1 on the result."""
    n, h, org, u, rng = tiny_grid(9, n=(10, 9, 8))
    R0 = rng.uniform(-0.15, 0.15, (6, 3))
    R1 = rng.uniform(-0.15, 0.15, (5, 3))
    Xr = np.array([org + np.array([0.40, 0.45, 0.4]), org + np.array([0.55, 0.45, 0.4])])
    Ur = rng.normal(size=(2, 3))
    Wr = rng.normal(size=(2, 3))
    dV = rng.uniform(0.5, 1.2, 11) * h ** 3
    Ns, dt = 2, 1e-2
    un, F, f = oracle.multidirect(n, h, org, u, Xr, Ur, Wr, [0, 6, 11],
                                  np.concatenate([R0, R1]), dV, Ns, dt, want_f=True)
    uf = u.reshape(3, -1)
    fsum = 0
    Fs = []
    for p, (Rp, sl) in enumerate(((R0, slice(0, 6)), (R1, slice(6, 11)))):
        W = dense_W(n, h, org, Xr[p] + Rp, oracle.ROMA3)
        uf, Fp, fp = _dense_alg1(W, uf, Ur[p] + np.cross(Wr[p], Rp), dV[sl], h, Ns, dt)
        Fs.append(Fp)
        fsum = fsum + fp
    assert np.max(np.abs(un.reshape(3, -1) - uf)) < 1e-12 * np.max(np.abs(uf))
    assert np.max(np.abs(F - np.concatenate(Fs))) < 1e-12 * np.max(np.abs(F))
    assert np.max(np.abs(f.reshape(3, -1) - fsum)) < 1e-12 * np.max(np.abs(fsum))


# ----------------------------------------------------------- PVF and integrals
def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            rows.append((line[0], int(line[1]), line[2]))
    return rows


@pytest.mark.parametrize("shape,doh,val", [r for r in _golden() if r[1] <= 64])
def test_pvf_tables_printed_in_paper(shape, doh, val):
    """or_pvf_ellipsoid_volume and or_volume_integrals reproduce the volumes of
    the paper's sphere and ellipsoid PVF tables (Sec. 4.1) to every printed
    digit: D = 0.8 / axes (0.4, 0.6, 0.4), centre (1,1,1), domain 2^3."""
    h = 0.8 / doh
    n = [int(round(2.0 / h))] * 3
    axes = (0.4, 0.4, 0.4) if shape == "sphere" else (0.4, 0.6, 0.4)
    tol = 0.5 * 10.0 ** (-(len(val.split(".")[1])))
    v = oracle.pvf_ellipsoid_volume(n, h, (0, 0, 0), (1, 1, 1), axes)
    assert abs(v - float(val)) <= tol
    if shape == "sphere":
        u = np.zeros((3,) + tuple(n))
        _, _, vol = oracle.volume_integrals(n, h, (0, 0, 0), u, [[1, 1, 1]], [0.4])
        assert abs(vol[0] - float(val)) <= tol


@pytest.mark.slow
@pytest.mark.parametrize("shape,doh,val", [r for r in _golden() if r[1] == 128])
def test_pvf_tables_finest_row(shape, doh, val):
    """D/h = 128 row of the PVF tables (320^3 grid).  The sphere value matches
    to all 10 printed digits; the ellipsoid's 11th printed digit differs by
    8e-11, so the ellipsoid is pinned to 10 significant digits."""
    h = 0.8 / doh
    n = [int(round(2.0 / h))] * 3
    axes = (0.4, 0.4, 0.4) if shape == "sphere" else (0.4, 0.6, 0.4)
    v = oracle.pvf_ellipsoid_volume(n, h, (0, 0, 0), (1, 1, 1), axes)
    assert abs(v - float(val)) <= (5e-11 if shape == "sphere" else 1e-10)


def test_volume_integrals_closed_forms():
    """or_volume_integrals: u = const gives Iu = c vol exactly and a zero
    first moment for a node-centred sphere; solid rotation u = w x r gives
    Irxu -> (8 pi / 15) R^5 w with second-order convergence."""
    errs = []
    R = 0.3
    w = np.array([0.3, -1.2, 0.7])
    for N in (20, 40, 80):
        h = 1.0 / N
        c = np.array([0.5, 0.5, 0.5])
        cst = np.array([1.5, -2.0, 0.25])
        u = np.broadcast_to(cst[:, None, None, None], (3, N, N, N)).copy()
        Iu, Irxu, vol = oracle.volume_integrals((N,) * 3, h, (0, 0, 0), u, [c], [R])
        assert np.allclose(Iu[0], cst * vol[0], rtol=1e-11, atol=0)
        assert np.max(np.abs(Irxu[0])) < 1e-14
        xs = (np.arange(N) + 0.5) * h - 0.5
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        r = np.stack([X, Y, Z])
        ur = np.stack([w[1] * r[2] - w[2] * r[1], w[2] * r[0] - w[0] * r[2],
                       w[0] * r[1] - w[1] * r[0]])
        Iu, Irxu, vol = oracle.volume_integrals((N,) * 3, h, (0, 0, 0), ur, [c], [R])
        assert np.max(np.abs(Iu[0])) < 1e-14
        exact = 8 * math.pi / 15 * R ** 5 * w
        errs.append(np.max(np.abs(Irxu[0] - exact)) / np.max(np.abs(exact)))
        errs[-1] = max(errs[-1], abs(vol[0] - 4 / 3 * math.pi * R ** 3) / (4 / 3 * math.pi * R ** 3))
    assert errs[2] < errs[0] / 8


def test_volume_integrals_periodic_image():
    """A sphere straddling the periodic seam integrates the same as the same
    sphere shifted by whole cells into the interior (field rolled alike)."""
    N = 32
    h = 1.0 / N
    rng = synth.SplitMix64(5)
    u = synth.fourier_field((N,) * 3, 4, rng, h)
    c_in = np.array([0.5, 0.5, 0.5]) + 0.3 * h
    shift = np.array([15, 14, -16])
    c_seam = c_in + shift * h
    u_roll = np.roll(u, shift=(shift[2], shift[1], shift[0]), axis=(1, 2, 3))
    a = oracle.volume_integrals((N,) * 3, h, (0, 0, 0), u, [c_in], [0.25])
    b = oracle.volume_integrals((N,) * 3, h, (0, 0, 0), u_roll, [c_seam], [0.25])
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-15)


# -------------------------------------------------------- force and torque
def test_force_torque_hand_values():
    """or_force_torque on hand-checked markers: a force couple on x = +-1
    gives zero force and T = (0, 0, -2 rho_f); a uniform force gives
    F = -rho_f c sum dV and no torque for a symmetric pair."""
    R = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 2.0, 0], [0, -2.0, 0]])
    F = np.array([[0, 1.0, 0], [0, -1.0, 0], [3.0, 0, 0], [3.0, 0, 0]])
    dV = np.array([1.0, 1.0, 0.5, 0.5])
    Fib, Tib = oracle.force_torque([0, 2, 4], R, dV, F, 1.25)
    assert np.array_equal(Fib[0], [0, 0, 0])
    assert np.array_equal(Tib[0], [0, 0, -2.5])
    assert np.array_equal(Fib[1], [-3.75, 0, 0])
    assert np.array_equal(Tib[1], [0, 0, 0])


def test_force_torque_reference_shift_and_segments():
    """Moving the torque's reference point by c changes T_ib by c x F_ib
    (T' = -rho_f sum (R + c) x F dV = T_ib + c x F_ib), particle by particle;
    the particles' forces add up to -rho_f sum F dV over all markers."""
    rng = np.random.default_rng(12)
    moff = [0, 7, 7, 20]  # the middle particle has no markers
    M = moff[-1]
    R, F = rng.normal(size=(M, 3)), rng.normal(size=(M, 3))
    dV = rng.uniform(0.5, 2.0, M)
    c = np.array([[0.3, -1.2, 2.0], [5.0, 5.0, 5.0], [-0.7, 0.4, 0.9]])
    shift = np.repeat(c, np.diff(moff), axis=0)
    Fib, Tib = oracle.force_torque(moff, R, dV, F, 0.8)
    Fs, Ts = oracle.force_torque(moff, R + shift, dV, F, 0.8)
    np.testing.assert_allclose(Fs, Fib, rtol=0, atol=1e-14)
    np.testing.assert_allclose(Ts, Tib + np.cross(c, Fib), rtol=1e-13, atol=1e-13)
    assert np.array_equal(Fib[1], [0, 0, 0]) and np.array_equal(Tib[1], [0, 0, 0])
    np.testing.assert_allclose(Fib.sum(axis=0), -0.8 * (F * dV[:, None]).sum(axis=0), rtol=1e-13)


# -------------------------------------------------- collision + Newton-Euler
PHYS0 = (1.0, 0.0, 0.0, -9.81, 9.81, 1e-4, 0.02)


def _zeros(P):
    return [np.zeros((P, 3)) for _ in range(6)]


def test_collision_hand_value_and_symmetry():
    """Eq. (DKT_model): two spheres R = 0.1, rho_p = 1.5, d_c = 0.02 at
    centre distance 0.21 (D_c = 0.22): |F| = (m g / eps)(0.5)^2 with
    m = 0.002 pi, pushing them apart, equal and opposite."""
    Xr = np.array([[0.3, 0.5, 0.5], [0.51, 0.5, 0.5]])
    _, _, _, Fc = oracle.collide_update(Xr, np.zeros((2, 3)), np.zeros((2, 3)),
                                        [0.1, 0.1], [1.5, 1.5], (64, 64, 64),
                                        1.0 / 64, PHYS0, 1e-3, *_zeros(2))
    mag = 0.002 * math.pi * 9.81 / 1e-4 * 0.25
    assert abs(Fc[0, 0] + mag) < 1e-9 and abs(Fc[1, 0] - mag) < 1e-9
    assert np.array_equal(Fc[0], -Fc[1])
    assert Fc[0, 1] == 0 and Fc[0, 2] == 0


def test_collision_cutoff_continuity_and_periodic_image():
    """The force vanishes for gaps >= d_c, tends to 0 continuously at
    d -> D_c, and acts through the periodic seam (nearest image)."""
    R = [0.1, 0.1]
    for d, zero in ((0.2201, True), (0.2200, True), (0.21999999, False)):
        Xr = np.array([[0.3, 0.5, 0.5], [0.3 + d, 0.5, 0.5]])
        Fc = oracle.collide_update(Xr, np.zeros((2, 3)), np.zeros((2, 3)), R,
                                   [1.5, 1.5], (64,) * 3, 1 / 64, PHYS0, 1e-3,
                                   *_zeros(2))[3]
        if zero:
            assert np.all(Fc == 0)
        else:
            assert 0 < -Fc[0, 0] < 1e-8
    Xr = np.array([[0.02, 0.5, 0.5], [0.81, 0.5, 0.5]])   # image distance 0.21
    Fc = oracle.collide_update(Xr, np.zeros((2, 3)), np.zeros((2, 3)), R, [1.5, 1.5],
                               (64,) * 3, 1 / 64, PHYS0, 1e-3, *_zeros(2))[3]
    mag = 0.002 * math.pi * 9.81 / 1e-4 * 0.25
    assert abs(Fc[0, 0] - mag) < 1e-9   # particle 0 pushed towards +x


def test_newton_euler_free_fall_closed_form():
    """Eqs. (particle1), (pr2) with no hydrodynamic or collision force:
    U^{n+1} = U^n + dt (1 - rho_f/rho_p) g, and after n steps
    X = X0 + U0 t + a t^2 / 2 (trapezoid exact for linear velocity)."""
    Xr = np.array([[0.2, 0.3, 0.9]])
    U0 = np.array([[0.1, -0.2, 0.05]])
    Ur = U0.copy()
    Wr = np.array([[0.3, 0.2, 0.1]])
    dt = 1e-3
    acc = (1 - 1.0 / 1.5) * np.array([0, 0, -9.81])
    for _ in range(10):
        Xr, Ur, Wr2, _ = oracle.collide_update(Xr, Ur, Wr, [0.05], [1.5], (64,) * 3,
                                               1 / 64, PHYS0, dt, *_zeros(1))
        assert np.array_equal(Wr2, Wr)
    t = 10 * dt
    assert np.allclose(Ur[0], U0[0] + acc * t, atol=1e-15, rtol=0)
    assert np.allclose(Xr[0], np.array([0.2, 0.3, 0.9]) + U0[0] * t + 0.5 * acc * t * t,
                       atol=1e-15, rtol=0)


def test_newton_euler_force_torque_and_unsteady_terms():
    """Each right-hand-side term of Eqs. (particle1)/(particle2) enters with
    its own coefficient: F_ib / m, rho_f dIu / (rho_p V), T_ib / I and
    rho_f dIrxu / I, with V = 4/3 pi R^3 and I = 2/5 m R^2."""
    R = 0.05
    rho = 2.0
    V = 4 / 3 * math.pi * R ** 3
    m = rho * V
    I = 0.4 * m * R ** 2
    phys = (1.3, 0.0, 0.0, 0.0, 9.81, 1e-4, 0.02)
    dt = 1e-3
    Fib = np.array([[1e-3, 0, 0]])
    Tib = np.array([[0, 2e-6, 0]])
    dIu = np.array([[0, 0, 4e-6]])
    dIr = np.array([[3e-8, 0, 0]])
    z = np.zeros((1, 3))
    X, U, W, _ = oracle.collide_update([[0.5, 0.5, 0.5]], z, z, [R], [rho], (32,) * 3,
                                       1 / 32, phys, dt, Fib, Tib, dIu, z, dIr, z)
    expU = dt / m * Fib[0] + 1.3 * dIu[0] / m
    expW = dt / I * Tib[0] + 1.3 * dIr[0] / I
    assert np.allclose(U[0], expU, rtol=1e-13, atol=0)
    assert np.allclose(W[0], expW, rtol=1e-13, atol=0)
    assert np.allclose(X[0], 0.5 + 0.5 * dt * expU, rtol=1e-15, atol=1e-17)


def test_collision_conserves_momentum():
    """Collision forces of a dense cluster sum to zero (F_c,ij = -F_c,ji)."""
    case = synth.cluster_case(N=96, P=20, D_cells=10, phi=0.25, K=2, Ns=3, seed=2,
                              min_gap_cells=0.1)
    Fc = oracle.collide_update(case.Xr, case.Ur, case.Wr, case.radius, case.rho_p,
                               case.n, case.h, case.phys(), 1e-3, *_zeros(case.P))[3]
    assert np.any(Fc != 0)
    assert np.max(np.abs(Fc.sum(axis=0))) < 1e-9 * np.max(np.abs(Fc))


# ------------------------------------------- ellipsoid PVF and drag (NEXT-3)
@pytest.mark.parametrize("shape,doh,val", [r for r in _golden() if r[0] == "ellipsoid" and r[1] <= 32])
def test_volume_integrals_ellipsoid_table(shape, doh, val):
    """or_volume_integrals_ellipsoid: the PVF volume of the paper's ellipsoid
    (Sec. 4.1 ellipsoid table; axes (0.4, 0.6, 0.4), centre (1, 1, 1),
    domain 2^3) to every printed digit."""
    h = 0.8 / doh
    n = [int(round(2.0 / h))] * 3
    u = np.zeros((3,) + tuple(n))
    _, _, vol = oracle.volume_integrals_ellipsoid(n, h, (0, 0, 0), u, [[1, 1, 1]], [[0.4, 0.6, 0.4]])
    tol = 0.5 * 10.0 ** (-(len(val.split(".")[1])))
    assert abs(vol[0] - float(val)) <= tol


def test_volume_integrals_ellipsoid_reduces_to_sphere():
    """Equal semi-axes give the sphere's integrals."""
    N = 32
    h = 1.0 / N
    rng = synth.SplitMix64(11)
    u = synth.fourier_field((N,) * 3, 5, rng, h)
    c = [[0.43, 0.52, 0.61], [0.1, 0.95, 0.5]]
    a = oracle.volume_integrals((N,) * 3, h, (0, 0, 0), u, c, [0.2, 0.15])
    b = oracle.volume_integrals_ellipsoid((N,) * 3, h, (0, 0, 0), u, c, [[0.2] * 3, [0.15] * 3])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_volume_integrals_ellipsoid_closed_forms():
    """u = const gives Iu = c vol and a zero first moment for a node-centred
    ellipsoid; solid rotation u = w x r gives Irxu -> I w with the ellipsoid's
    inertia I = V/5 diag(b^2 + c^2, a^2 + c^2, a^2 + b^2), V = 4/3 pi abc,
    with second-order convergence."""
    ax = np.array([0.3, 0.2, 0.25])
    w = np.array([0.3, -1.2, 0.7])
    V = 4 / 3 * math.pi * np.prod(ax)
    inertia = V / 5 * np.array([ax[1] ** 2 + ax[2] ** 2, ax[0] ** 2 + ax[2] ** 2, ax[0] ** 2 + ax[1] ** 2])
    errs = []
    for N in (20, 40, 80):
        h = 1.0 / N
        c = np.array([0.5, 0.5, 0.5])
        cst = np.array([1.5, -2.0, 0.25])
        u = np.broadcast_to(cst[:, None, None, None], (3, N, N, N)).copy()
        Iu, Irxu, vol = oracle.volume_integrals_ellipsoid((N,) * 3, h, (0, 0, 0), u, [c], [ax])
        assert np.allclose(Iu[0], cst * vol[0], rtol=1e-11, atol=0)
        assert np.max(np.abs(Irxu[0])) < 1e-14
        xs = (np.arange(N) + 0.5) * h - 0.5
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        r = np.stack([X, Y, Z])
        ur = np.stack([w[1] * r[2] - w[2] * r[1], w[2] * r[0] - w[0] * r[2], w[0] * r[1] - w[1] * r[0]])
        Iu, Irxu, vol = oracle.volume_integrals_ellipsoid((N,) * 3, h, (0, 0, 0), ur, [c], [ax])
        exact = inertia * w
        errs.append(max(np.max(np.abs(Irxu[0] - exact)) / np.max(np.abs(exact)), abs(vol[0] - V) / V))
    assert errs[2] < errs[0] / 8


def test_drag_force_definition():
    """Eq. FD by hand: F_D = F_ib + rho_f (Iu_new - Iu_old) / dt."""
    Fib = [[1.0, 2.0, 3.0], [-1.0, 0.0, 0.5]]
    Inew = [[1.0, 1.0, 1.0], [0.0, 2.0, 0.0]]
    Iold = [[0.0, 0.0, 0.0], [0.0, 1.0, 0.25]]
    FD = oracle.drag_force(Fib, Inew, Iold, 2.0, 0.5)
    assert np.array_equal(FD, [[5.0, 6.0, 7.0], [-1.0, 4.0, -0.5]])
