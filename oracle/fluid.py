"""FP64 oracle of the fluid step around the IB forcing (test infrastructure).

Only the tests, the smoke check and the bench's CPU-baseline leg use this
module; the library never imports it.  It restates Step 1 (the momentum
predictor, Eq. 31) and Step 3 (the level projection, Eqs. ns_lp1-ns_lp3) of
Sec. 3.1 on one uniform periodic level, in numpy, with numpy's FFT as the
only library step.

Grid (Sec. 3.1, semi-staggered grid): n0 x n1 x n2 cells of size h, periodic.
Velocity components sit at cell centres (i + 1/2) h and are stored
[3][n2][n1][n0] (x fastest); the pressure sits at nodes i h and is stored
[n2][n1][n0], node (i, j, k) being the lower corner of cell (i, j, k).

Readings where the paper defers to its cited solver (all listed in the
design notes):
* gradient of a nodal field at a cell centre: the four node differences
  across the cell along the axis, averaged;
* divergence of a cell field at a node: the negative adjoint of that
  gradient, so that the projection's Laplacian is exactly D G;
* the level projection solves D G p = rho D V exactly by FFT; the Fourier
  modes where the symbol of D G vanishes (the mean and the nodal checkerboard
  modes, which D cannot produce) get p = 0;
* viscosity by Crank-Nicolson with the 7-point cell Laplacian, its implicit
  half solved exactly by FFT;
* the convective term by a second-order Godunov edge extrapolation: per
  face, states from both neighbours by a Taylor step of (h/2 -+ dt u_n/2)
  along monotonized-central limited slopes, the normal face velocity from
  the Burgers Riemann solution of the two normal states, the transported
  state upwinded by it (the average of both when it is zero), and the flux
  divergence of u_face (x) s_face; no transverse terms, no MAC projection.
"""
from __future__ import annotations

import numpy as np

AX = {0: -1, 1: -2, 2: -3}  # grid axis -> numpy axis of a [..., n2, n1, n0] array


def _sh(a, axis, k):
    """a shifted so that element i holds a[i + k] along grid axis `axis` (periodic)."""
    return np.roll(a, -k, axis=AX[axis])


def grad_node_to_cell(p, h):
    """G p at cell centres: along x, (1/4h) sum over the cell's four x-edges of
    p(i+1, .) - p(i, .), i.e. the node differences at (j|j+1, k|k+1)."""
    out = np.empty((3,) + p.shape)
    for a in range(3):
        d = _sh(p, a, 1) - p                      # difference along a, at the node (i, j, k)
        b, c = [x for x in range(3) if x != a]
        out[a] = 0.25 / h * (d + _sh(d, b, 1) + _sh(d, c, 1) + _sh(_sh(d, b, 1), c, 1))
    return out


def div_cell_to_node(V, h):
    """D V at nodes, the negative adjoint of grad_node_to_cell: along x,
    (1/4h) sum over the four cell pairs around the node of V(i) - V(i-1)."""
    out = np.zeros(V.shape[1:])
    for a in range(3):
        d = V[a] - _sh(V[a], a, -1)               # across the node along a, for the cells (j|j-1, k|k-1)
        b, c = [x for x in range(3) if x != a]
        out += 0.25 / h * (d + _sh(d, b, -1) + _sh(d, c, -1) + _sh(_sh(d, b, -1), c, -1))
    return out


def lap_cell(u, h):
    """7-point Laplacian of each cell-centred component."""
    out = np.zeros_like(u)
    for a in range(3):
        out += (_sh(u, a, 1) - 2.0 * u + _sh(u, a, -1)) / (h * h)
    return out


def _theta(shape):
    """theta_a = 2 pi k_a / n_a on the FFT grid of a [n2, n1, n0] array, as
    (theta_x, theta_y, theta_z) broadcast to the shape."""
    n2, n1, n0 = shape
    tz = 2 * np.pi * np.fft.fftfreq(n2)[:, None, None]
    ty = 2 * np.pi * np.fft.fftfreq(n1)[None, :, None]
    tx = 2 * np.pi * np.fft.fftfreq(n0)[None, None, :]
    return tx, ty, tz


def symbol_lap_cell(shape, h):
    """Fourier symbol of lap_cell: -(4/h^2) sum_a sin^2(theta_a / 2)."""
    tx, ty, tz = _theta(shape)
    return -(4.0 / (h * h)) * (np.sin(tx / 2) ** 2 + np.sin(ty / 2) ** 2 + np.sin(tz / 2) ** 2)


def symbol_div_grad(shape, h):
    """Fourier symbol of D G: -(4/h^2) sum_a sin^2(theta_a/2) prod_(b != a) cos^2(theta_b/2)."""
    tx, ty, tz = _theta(shape)
    sx, sy, sz = np.sin(tx / 2) ** 2, np.sin(ty / 2) ** 2, np.sin(tz / 2) ** 2
    cx, cy, cz = np.cos(tx / 2) ** 2, np.cos(ty / 2) ** 2, np.cos(tz / 2) ** 2
    return -(4.0 / (h * h)) * (sx * cy * cz + sy * cx * cz + sz * cx * cy)


def solve_div_grad(rhs, h):
    """p with D G p = rhs (periodic, FFT); modes where the symbol vanishes get
    p = 0.  The symbol is real and even, so p is real."""
    lam = symbol_div_grad(rhs.shape, h)
    r = np.fft.fftn(rhs)
    scale = np.max(np.abs(lam))
    null = np.abs(lam) <= 1e-13 * scale
    ph = np.where(null, 0.0, r / np.where(null, 1.0, lam))
    return np.real(np.fft.ifftn(ph))


def solve_helmholtz(rhs, coef, h):
    """x with (I - coef lap_cell) x = rhs per component (periodic, FFT)."""
    lam = 1.0 - coef * symbol_lap_cell(rhs.shape[1:], h)
    out = np.empty_like(rhs)
    for a in range(rhs.shape[0]):
        out[a] = np.real(np.fft.ifftn(np.fft.fftn(rhs[a]) / lam))
    return out


def _mc_slope(um, u0, up):
    """Monotonized-central limited difference of u0 from its neighbours."""
    a, b = u0 - um, up - u0
    mag = np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(b)), 0.5 * np.abs(a + b))
    return np.where(a * b > 0, np.sign(a + b) * mag, 0.0)


def convection(u, h, dt):
    """div(u u)^{n+1/2} at cell centres by the Godunov edge extrapolation of
    the module docstring: for each axis a and the face between cells i and
    i+1 along a, every component c gets the states
      left  = u_c(i)   + (1/2 - dt u_a(i)   / (2h)) slope_c(i)
      right = u_c(i+1) - (1/2 + dt u_a(i+1) / (2h)) slope_c(i+1),
    the face velocity is the Burgers Riemann solution of (left_a, right_a),
    and the flux u_face * state(upwind) differences over the cell."""
    out = np.zeros_like(u)
    for a in range(3):
        slope = np.stack([_mc_slope(_sh(u[c], a, -1), u[c], _sh(u[c], a, 1)) for c in range(3)])
        ua = u[a]
        left = u + (0.5 - dt * ua / (2 * h)) * slope                                   # at face i+1/2 from i
        right = _sh(u, a, 1) - (0.5 + dt * _sh(ua, a, 1) / (2 * h)) * _sh(slope, a, 1)  # from i+1
        lv, rv = left[a], right[a]
        un = np.where((lv > 0) & (lv + rv > 0), lv, np.where((rv < 0) & (lv + rv < 0), rv, 0.0))
        state = np.where(un > 0, left, np.where(un < 0, right, 0.5 * (left + right)))
        flux = un * state                                                            # face i+1/2
        out += (flux - _sh(flux, a, -1)) / h
    return out


def predictor(u, p, rho_f, mu, g, dt, h):
    """Step 1, Eq. 31: the intermediate velocity u~*,n+1 from
    rho_f ((u~* - u^n)/dt + div(u u)^{n+1/2}) = -grad p^{n-1/2}
        + (1/2)(div mu grad u~* + div mu grad u^n) + rho_f g,
    i.e. (I - (nu dt/2) L) u~* = u^n + dt (-div(u u) - G p / rho_f + (nu/2) L u^n + g)
    with nu = mu / rho_f."""
    nu = mu / rho_f
    rhs = u + dt * (-convection(u, h, dt) - grad_node_to_cell(p, h) / rho_f + 0.5 * nu * lap_cell(u, h)
                    + np.asarray(g, float)[:, None, None, None])
    return solve_helmholtz(rhs, 0.5 * nu * dt, h)


def projection(u_star, p_old, rho_f, dt, h):
    """Step 3: V = u*/dt + (1/rho_f) grad p^{n-1/2} (Eq. ns_lp1);
    L p^{n+1/2} = div V with L p = div((1/rho_f) grad p) (Eq. ns_lp2);
    u^{n+1} = dt (V - (1/rho_f) grad p^{n+1/2}) (Eq. ns_lp3).
    Returns (u^{n+1}, p^{n+1/2})."""
    V = u_star / dt + grad_node_to_cell(p_old, h) / rho_f
    p_new = rho_f * solve_div_grad(div_cell_to_node(V, h), h)
    u_new = dt * (V - grad_node_to_cell(p_new, h) / rho_f)
    return u_new, p_new
