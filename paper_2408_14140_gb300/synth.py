"""Seeded synthetic inputs shaped like the paper's particle-laden cases.

This module produces INPUTS only -- grids, velocity fields, particle
placements and surface-marker templates -- and holds none of the method's
arithmetic (no delta kernel, interpolation, spreading, forcing, PVF or
collision law).  The same arrays feed the CUDA library and the FP64 oracle.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) with
Box-Muller normals, so every case is reproducible from its seed on any host.

Recipe (shapes of the paper's cases; no dataset is involved):
  * unit periodic domain, h = 1/N, cell-centred grid, origin 0;
  * velocity u(x) = sum_k a_k cos(2 pi n_k . x / L + theta_k), a_k ~ N(0,1)^3,
    n_k integer with components uniform in [-4, 4], n_k != 0,
    theta_k ~ U[0, 2 pi);
  * spheres of diameter D cells carry N_L = round(pi (D/h)^2) markers on a
    Fibonacci lattice, i.e. about one marker per h^2 of surface (the surface
    marker layout of Sec. 3.1 Step 2);
  * each marker carries the volume of a shell of thickness h divided evenly,
    dV = (pi h / 3)(12 R^2 + h^2) / N_L  (the paper leaves dV unstated);
  * particle velocities U_r, W_r ~ N(0, 0.1^2) per component;
  * monodisperse spheres are placed by random sequential addition without
    overlap inside a centred cluster box sized for the requested volume
    fraction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``uniform`` in [0,1) from the top 53 bits."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, k: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(k)])

    def normal(self) -> float:
        u1 = self.uniform()
        while u1 <= 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)

    def normals(self, k: int) -> np.ndarray:
        return np.array([self.normal() for _ in range(k)])

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))


# --------------------------------------------------------------------------
# markers
# --------------------------------------------------------------------------

def fibonacci_sphere(NL: int) -> np.ndarray:
    """NL unit vectors on a Fibonacci lattice, [NL, 3]."""
    l = np.arange(NL, dtype=np.float64)
    z = 1.0 - (2.0 * l + 1.0) / NL
    theta = l * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(theta), r * np.sin(theta), z], axis=1)


def markers_per_sphere(D_cells: float) -> int:
    return int(round(math.pi * D_cells * D_cells))


def sphere_markers(radius: float, h: float):
    """(R[NL,3] offsets from the centre, dV[NL]) for one sphere."""
    NL = markers_per_sphere(2.0 * radius / h)
    R = radius * fibonacci_sphere(NL)
    dv = (math.pi * h / 3.0) * (12.0 * radius * radius + h * h) / NL
    return R, np.full(NL, dv)


# --------------------------------------------------------------------------
# fields
# --------------------------------------------------------------------------

def fourier_modes(K: int, rng: SplitMix64):
    """K random modes (a_k[3], n_k[3] integers, theta_k) in draw order."""
    modes = []
    for _ in range(K):
        a = rng.normals(3)
        while True:
            kv = [rng.randint(-4, 4) for _ in range(3)]
            if any(kv):
                break
        th = 2.0 * math.pi * rng.uniform()
        modes.append((a, kv, th))
    return modes


def fourier_eval(n, modes, h, org=(0.0, 0.0, 0.0), dtype=np.float64) -> np.ndarray:
    """u[3, n2, n1, n0] = sum_k a_k cos(2 pi n_k . x / L + theta_k) at cell centres."""
    n = [int(v) for v in n]
    L = [n[a] * h for a in range(3)]
    xs = [org[a] + (np.arange(n[a]) + 0.5) * h for a in range(3)]
    u = np.zeros((3, n[2], n[1], n[0]), dtype=np.float64)
    for a, kv, th in modes:
        ex = np.exp(1j * 2.0 * math.pi * kv[0] * xs[0] / L[0])
        ey = np.exp(1j * 2.0 * math.pi * kv[1] * xs[1] / L[1])
        ez = np.exp(1j * (2.0 * math.pi * kv[2] * xs[2] / L[2] + th))
        for k0 in range(0, n[2], 32):
            blk = (ez[k0:k0 + 32, None, None] * ey[None, :, None]
                   * ex[None, None, :]).real
            for c in range(3):
                u[c, k0:k0 + 32] += a[c] * blk
    return u.astype(dtype, copy=False)


def fourier_eval_torch(n, modes, h, org=(0.0, 0.0, 0.0), device="cuda", dtype=None):
    """Same field as :func:`fourier_eval`, evaluated with torch on ``device``
    (FP64 arithmetic, then cast) -- used for grids too large to build on the
    host quickly."""
    import torch
    n = [int(v) for v in n]
    L = [n[a] * h for a in range(3)]
    xs = [org[a] + (torch.arange(n[a], device=device, dtype=torch.float64) + 0.5) * h
          for a in range(3)]
    u = torch.zeros((3, n[2], n[1], n[0]), device=device, dtype=torch.float64)
    for a, kv, th in modes:
        ex = torch.exp(1j * 2.0 * math.pi * kv[0] * xs[0] / L[0])
        ey = torch.exp(1j * 2.0 * math.pi * kv[1] * xs[1] / L[1])
        ez = torch.exp(1j * (2.0 * math.pi * kv[2] * xs[2] / L[2] + th))
        blk = (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).real
        for c in range(3):
            u[c] += float(a[c]) * blk
        del blk
    return u if dtype is None else u.to(dtype)


def fourier_field(n, K: int, rng: SplitMix64, h: float | None = None,
                  org=(0.0, 0.0, 0.0), dtype=np.float64) -> np.ndarray:
    """u[3, n2, n1, n0] = sum of K random Fourier modes at cell centres."""
    if h is None:
        h = 1.0 / int(n[0])
    return fourier_eval(n, fourier_modes(K, rng), h, org, dtype)


def taylor_green_field(n, U0: float = 1.0, h: float | None = None,
                       org=(0.0, 0.0, 0.0), dtype=np.float64) -> np.ndarray:
    """Steady Taylor-Green vortex on the unit periodic cube."""
    n = [int(v) for v in n]
    if h is None:
        h = 1.0 / n[0]
    x = org[0] + (np.arange(n[0]) + 0.5) * h
    y = org[1] + (np.arange(n[1]) + 0.5) * h
    z = org[2] + (np.arange(n[2]) + 0.5) * h
    tp = 2.0 * math.pi
    sx, cx = np.sin(tp * x), np.cos(tp * x)
    sy, cy = np.sin(tp * y), np.cos(tp * y)
    cz = np.cos(tp * z)
    u = np.zeros((3, n[2], n[1], n[0]))
    u[0] = U0 * cz[:, None, None] * cy[None, :, None] * sx[None, None, :]
    u[1] = -U0 * cz[:, None, None] * sy[None, :, None] * cx[None, None, :]
    return u.astype(dtype, copy=False)


# --------------------------------------------------------------------------
# particles
# --------------------------------------------------------------------------

def rsa_place(P: int, D: float, box_lo, box_hi, min_gap: float,
              rng: SplitMix64, max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential addition of P spheres of diameter D (centres kept at
    least D/2 from the box faces and D + min_gap apart).  [P, 3]."""
    lo = np.asarray(box_lo, dtype=np.float64) + 0.5 * D
    hi = np.asarray(box_hi, dtype=np.float64) - 0.5 * D
    cent = np.zeros((P, 3))
    dmin2 = (D + min_gap) ** 2
    placed = 0
    tries = 0
    while placed < P:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rsa_place: could not place %d spheres" % P)
        c = lo + (hi - lo) * rng.uniforms(3)
        if placed:
            d2 = np.sum((cent[:placed] - c) ** 2, axis=1)
            if np.any(d2 < dmin2):
                continue
        cent[placed] = c
        placed += 1
    return cent


@dataclass
class Case:
    """One periodic IB case: grid, field, particles and markers (numpy)."""
    n: tuple
    h: float
    org: tuple
    u: np.ndarray              # [3, n2, n1, n0] float64
    Xr: np.ndarray             # [P, 3]
    Ur: np.ndarray
    Wr: np.ndarray
    radius: np.ndarray         # [P]
    rho_p: np.ndarray          # [P]
    moff: np.ndarray           # [P+1] int64
    R: np.ndarray              # [M, 3]
    dV: np.ndarray             # [M]
    Ns: int = 3
    dt: float = 1e-3
    rho_f: float = 1.0
    g: tuple = (0.0, 0.0, -9.81)
    g_coll: float = 9.81
    eps_c: float = 1e-4
    d_c: float = 0.0           # set to h by the builders
    meta: dict = field(default_factory=dict)

    @property
    def P(self) -> int:
        return int(self.Xr.shape[0])

    @property
    def M(self) -> int:
        return int(self.moff[-1])

    def phys(self):
        return (self.rho_f, self.g[0], self.g[1], self.g[2], self.g_coll,
                self.eps_c, self.d_c)


def _assemble(n, h, u, cent, radii, rng, Ns, dt, rho_p=1.5, meta=None):
    P = cent.shape[0]
    Rs, dVs, moff = [], [], [0]
    for p in range(P):
        R, dv = sphere_markers(float(radii[p]), h)
        Rs.append(R)
        dVs.append(dv)
        moff.append(moff[-1] + R.shape[0])
    Ur = 0.1 * rng.normals(3 * P).reshape(P, 3)
    Wr = 0.1 * rng.normals(3 * P).reshape(P, 3)
    return Case(n=tuple(int(v) for v in n), h=h, org=(0.0, 0.0, 0.0), u=u,
                Xr=cent, Ur=Ur, Wr=Wr, radius=np.asarray(radii, float),
                rho_p=np.full(P, float(rho_p)),
                moff=np.asarray(moff, dtype=np.int64),
                R=np.concatenate(Rs) if Rs else np.zeros((0, 3)),
                dV=np.concatenate(dVs) if dVs else np.zeros(0),
                Ns=Ns, dt=dt, d_c=h, meta=meta or {})


def single_sphere_case(N: int = 64, D_cells: float = 20.0, K: int = 8,
                       Ns: int = 2, dt: float = 1e-3, seed: int = 0,
                       centre=None) -> Case:
    """One sphere of D cells centred in an N^3 periodic grid, K Fourier modes
    (the 64^3, D = 20, Ns = 2 correctness case)."""
    rng = SplitMix64(seed)
    h = 1.0 / N
    u = fourier_field((N, N, N), K, rng, h)
    c = np.array([[0.5, 0.5, 0.5]]) if centre is None else np.asarray(centre, float).reshape(1, 3)
    return _assemble((N, N, N), h, u, c, [0.5 * D_cells * h], rng, Ns, dt,
                     meta={"workload": "single-sphere", "N": N, "D": D_cells})


def cluster_case(N: int, P: int, D_cells: float, phi: float, K: int, Ns: int,
                 dt: float = 1e-3, seed: int = 0, min_gap_cells: float = 0.0,
                 u_dtype=np.float64, build_field: bool = True) -> Case:
    """P monodisperse spheres placed by RSA inside a centred cubic cluster box
    whose side makes their volume fraction ``phi`` (the 256^3 / 64 x D24 and
    384^3 / 512 x D16 cases)."""
    rng = SplitMix64(seed)
    h = 1.0 / N
    vsph = math.pi / 6.0 * D_cells ** 3
    side = (P * vsph / phi) ** (1.0 / 3.0)
    if side > N - 2:
        raise ValueError("cluster box does not fit the grid")
    lo = 0.5 * (N - side)
    cent = rsa_place(P, D_cells, [lo] * 3, [lo + side] * 3, min_gap_cells, rng)
    modes = fourier_modes(K, rng)
    u = fourier_eval((N, N, N), modes, h).astype(u_dtype, copy=False) if build_field else None
    case = _assemble((N, N, N), h, u, cent * h,
                     [0.5 * D_cells * h] * P, rng, Ns, dt,
                     meta={"workload": "cluster", "N": N, "P": P,
                           "D": D_cells, "phi": phi, "box_side": side,
                           "modes": modes})
    return case


def random_case(N: int, P: int, D_lo: float, D_hi: float, K: int, Ns: int,
                rng: SplitMix64, dt: float = 1e-3, field_kind: str = "fourier",
                min_gap_cells: float = 0.25, max_tries: int = 200) -> Case:
    """Polydisperse case: P spheres, D ~ U[D_lo, D_hi] cells, placed without
    overlap anywhere in the periodic box (redraw D, then the count, on
    failure).  Used by the batched and served workloads.  ``field_kind``:
    "fourier" (K modes, built on the host), "fourier-modes" (the same modes
    drawn, kept in ``meta["modes"]`` for evaluation on the device, no host
    field), "tgv" (Taylor-Green vortex) or "none"."""
    h = 1.0 / N
    for _ in range(max_tries):
        D = D_lo + (D_hi - D_lo) * rng.uniforms(P)
        if np.max(D) > N - 4:
            continue
        cent = np.zeros((P, 3))
        ok = True
        for p in range(P):
            lim = 0.5 * (D[p] + D[:p]) + min_gap_cells
            for _t in range(5000):
                c = rng.uniforms(3) * N
                d = c - cent[:p]
                d -= N * np.round(d / N)
                if p == 0 or np.all(np.sqrt(np.sum(d * d, axis=1)) >= lim):
                    cent[p] = c
                    break
            else:
                ok = False
                break
        if ok:
            break
        P = max(1, P - 1)
    else:
        raise RuntimeError("random_case: placement failed")
    meta = {"workload": "random", "N": N, "P": P}
    u = None
    if field_kind == "tgv":
        u = taylor_green_field((N, N, N), 1.0, h)
    elif field_kind == "fourier":
        u = fourier_field((N, N, N), K, rng, h)
    elif field_kind == "fourier-modes":
        meta["modes"] = fourier_modes(K, rng)
    elif field_kind != "none":
        raise ValueError("field_kind: " + field_kind)
    return _assemble((N, N, N), h, u, cent * h, 0.5 * D * h, rng, Ns, dt, meta=meta)


def taylor_green_torch(n, U0: float = 1.0, h: float | None = None, device="cuda", dtype=None):
    """:func:`taylor_green_field` evaluated with torch on ``device``."""
    import torch
    n = [int(v) for v in n]
    if h is None:
        h = 1.0 / n[0]
    xs = [(torch.arange(n[a], device=device, dtype=torch.float64) + 0.5) * h for a in range(3)]
    tp = 2.0 * math.pi
    sx, cx = torch.sin(tp * xs[0]), torch.cos(tp * xs[0])
    sy, cy = torch.sin(tp * xs[1]), torch.cos(tp * xs[1])
    cz = torch.cos(tp * xs[2])
    u = torch.zeros((3, n[2], n[1], n[0]), device=device, dtype=torch.float64)
    u[0] = U0 * cz[:, None, None] * cy[None, :, None] * sx[None, None, :]
    u[1] = -U0 * cz[:, None, None] * sy[None, :, None] * cx[None, None, :]
    return u if dtype is None else u.to(dtype)


def batched_cases(ncases: int = 256, seed: int = 0, grids=(32, 48, 64, 96, 128), P_max: int = 8,
                  D_lo: float = 8.0, D_hi: float = 24.0, K: int = 8, Ns: int = 3,
                  dt: float = 1e-3):
    """Independent periodic cases of the batched workload: grids drawn
    uniformly from ``grids`` (cubic), 1..P_max spheres each with D uniform in
    [D_lo, D_hi] cells, K Fourier modes per case (kept in meta["modes"]; the
    fields are evaluated on the device)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(ncases):
        N = int(grids[rng.randint(0, len(grids) - 1)])
        P = rng.randint(1, P_max)
        out.append(random_case(N, P, D_lo, D_hi, K, Ns, rng, dt, field_kind="fourier-modes"))
    return out
