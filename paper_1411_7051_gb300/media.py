"""Seeded synthetic porous media (porosity, intrinsic permeability, Kn).

These generators are the single source of inputs for the CUDA library, the
FP64 oracle, the tests and the benchmark.  They hold none of the lattice
Boltzmann arithmetic: they only draw fields.  Every array is row-major
[ny][nx] float64 (x fastest), in lattice units.

The paper's own geometries (Section IV.B: overlapping tolerance circles and
QSGS; Section IV.C: a shale image from the literature with tree-like
fractures) are not available, so statistically shaped stand-ins are drawn:

* ``channel``: the parallel-plate validation of Section IV.A (Eq. 18-20).
* ``two_component``: a thresholded Gaussian random field with a matrix phase
  and an inclusion phase (Section IV.B's heterogeneous medium).
* ``shale_fractures``: a low-porosity matrix with straight fractures
  (Section IV.C), with Kn set from the local pressure of a linear pressure
  drop and the pore radius scaling r ~ sqrt(k / eps) of Eq. 11.
* ``random_medium``: i.i.d. node values for parity tests, optionally with
  open pores (eps = 1, k = inf) and impermeable nodes (eps = 0).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Medium:
    eps: np.ndarray
    k_i: np.ndarray
    kn: np.ndarray
    name: str = ""

    @property
    def shape(self):
        return self.eps.shape

    def crop(self, ny: int, nx: int, y0: int = 0, x0: int = 0) -> "Medium":
        s = (slice(y0, y0 + ny), slice(x0, x0 + nx))
        return Medium(self.eps[s].copy(), self.k_i[s].copy(), self.kn[s].copy(),
                      f"{self.name}[{ny}x{nx}]")


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def channel(nx: int = 64, ny: int = 33, eps: float = 0.7, darcy: float = 1e-3,
            kn: float = 0.1) -> Medium:
    """Homogeneous medium between plates.  With wall rows 0 and ny-1 and
    halfway bounce-back the plate gap is H = ny - 2; k_i = darcy * H^2."""
    H = ny - 2
    shape = (ny, nx)
    return Medium(np.full(shape, float(eps)), np.full(shape, darcy * H * H),
                  np.full(shape, float(kn)), f"channel{nx}x{ny}")


def gaussian_field(ny: int, nx: int, corr_len: float, rng: np.random.Generator):
    """Periodic Gaussian random field with covariance exp(-r^2 / (2 L^2)):
    white noise filtered by a Gaussian of standard deviation L / sqrt(2)."""
    noise = rng.standard_normal((ny, nx))
    ky = np.fft.fftfreq(ny)[:, None] * 2 * np.pi
    kx = np.fft.fftfreq(nx)[None, :] * 2 * np.pi
    sigma = corr_len / np.sqrt(2.0)
    filt = np.exp(-0.5 * (kx * kx + ky * ky) * sigma * sigma)
    return np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))


def two_component(n: int = 1024, seed: int = 2, corr_len: float = 32.0,
                  kn: float = 0.1, matrix=(0.2, 1e-5), inclusion=(0.6, 1e-3),
                  ny: int | None = None) -> Medium:
    """Matrix / inclusion medium: a Gaussian random field thresholded at its
    median (exactly half of the nodes in each phase)."""
    ny = n if ny is None else ny
    g = gaussian_field(ny, n, corr_len, _rng(seed))
    inc = g > np.median(g)
    eps = np.where(inc, inclusion[0], matrix[0]).astype(np.float64)
    k_i = np.where(inc, inclusion[1], matrix[1]).astype(np.float64)
    return Medium(eps, k_i, np.full((ny, n), float(kn)), f"two_component{n}s{seed}")


def shale_fractures(n: int = 4096, seed: int = 3, n_fractures: int = 40,
                    kn_inlet: float = 0.5, p_out_over_p_in: float = 0.5,
                    length=(200.0, 2000.0), widths=(2, 3, 4),
                    fracture=(0.9, 1e-2)) -> Medium:
    """Shale matrix with straight fractures.

    Matrix: eps ~ U(0.05, 0.1), log10 k_i ~ N(-6, 0.3), i.i.d. per node.
    Fractures: centre uniform, angle U(0, pi), length U(length), width drawn
    from ``widths``; nodes within width/2 of the segment get ``fracture``.
    Kn: Kn = kn_inlet * (p_in / p(x)) * (r_ref / r), with p falling linearly
    from p_in at x = 0 to p_out at x = n-1 (mean free path ~ 1/p, Eq. 10) and
    r ~ sqrt(k_i / eps) (Eq. 11) normalised at the matrix median
    (k_i = 1e-6, eps = 0.075).
    """
    rng = _rng(seed)
    eps = rng.uniform(0.05, 0.1, size=(n, n))
    k_i = 10.0 ** rng.normal(-6.0, 0.3, size=(n, n))
    for _ in range(n_fractures):
        cx, cy = rng.uniform(0, n), rng.uniform(0, n)
        ang = rng.uniform(0, np.pi)
        L = rng.uniform(*length)
        w = int(rng.choice(widths))
        dx, dy = np.cos(ang), np.sin(ang)
        x0, y0 = cx - 0.5 * L * dx, cy - 0.5 * L * dy
        # bounding box of the segment
        xa = int(max(0, np.floor(min(x0, x0 + L * dx) - w)))
        xb = int(min(n, np.ceil(max(x0, x0 + L * dx) + w) + 1))
        ya = int(max(0, np.floor(min(y0, y0 + L * dy) - w)))
        yb = int(min(n, np.ceil(max(y0, y0 + L * dy) + w) + 1))
        if xa >= xb or ya >= yb:
            continue
        yy, xx = np.mgrid[ya:yb, xa:xb]
        px = xx - x0
        py = yy - y0
        t = np.clip(px * dx + py * dy, 0.0, L)
        d2 = (px - t * dx) ** 2 + (py - t * dy) ** 2
        mask = d2 <= (0.5 * w) ** 2
        eps[ya:yb, xa:xb][mask] = fracture[0]
        k_i[ya:yb, xa:xb][mask] = fracture[1]
    x = np.arange(n, dtype=np.float64)
    p_ratio = 1.0 - (1.0 - p_out_over_p_in) * x / (n - 1)  # p(x) / p_in
    r_ref = np.sqrt(1e-6 / 0.075)
    r = np.sqrt(k_i / eps)
    kn = kn_inlet * (1.0 / p_ratio)[None, :] * (r_ref / r)
    return Medium(eps, k_i, kn, f"shale{n}s{seed}")


def random_medium(nx: int, ny: int, seed: int, eps_range=(0.1, 1.0),
                  log10_k_range=(-4.0, 0.0), kn_range=(0.0, 10.0),
                  p_open: float = 0.0, p_solid: float = 0.0) -> Medium:
    """i.i.d. node values; a fraction ``p_open`` of nodes are open pores
    (eps = 1, k_i = inf) and ``p_solid`` impermeable nodes (eps = 0)."""
    rng = _rng(seed)
    eps = rng.uniform(*eps_range, size=(ny, nx))
    k_i = 10.0 ** rng.uniform(*log10_k_range, size=(ny, nx))
    kn = rng.uniform(*kn_range, size=(ny, nx))
    u = rng.uniform(size=(ny, nx))
    open_ = u < p_open
    solid = (u >= p_open) & (u < p_open + p_solid)
    eps[open_] = 1.0
    k_i[open_] = np.inf
    eps[solid] = 0.0
    return Medium(eps, k_i, kn, f"random{nx}x{ny}s{seed}")


def random_populations(nx: int, ny: int, seed: int, base, amp: float = 1e-3) -> np.ndarray:
    """Populations base_i (1 + amp * U(-1, 1)) in plane-major [9][ny][nx], for
    starting parity runs away from rest.  ``base`` (length 9) is supplied by
    the caller, e.g. the rest equilibrium of the lattice in use."""
    rng = _rng(seed)
    base = np.asarray(base, dtype=np.float64).reshape(9, 1, 1)
    return base * (1.0 + amp * rng.uniform(-1, 1, size=(9, ny, nx)))


PORE, IMPERMEABLE, PERMEABLE = 0, 1, 2


def trimodal(nx: int = 410, ny: int = 200, seed: int = 4, frac_solid: float = 0.4,
             frac_perm: float = 0.3, r_range=(4.0, 12.0), core_prob: float = 0.004,
             grow_axis: float = 0.02, grow_diag: float = 0.005) -> np.ndarray:
    """Labels of a three-component medium like that of Section IV.B (Fig. 4):
    PORE, IMPERMEABLE solid, PERMEABLE solid, as int8 [ny][nx].

    Impermeable solids: overlapping discs of radius U(r_range) with uniform
    centres (periodic wrap) until they cover frac_solid of the lattice.
    Permeable solids: quartet structure generation set (QSGS) in the space
    left: each free cell becomes a growth core with probability core_prob;
    then, sweep after sweep, every free cell next to a permeable one turns
    permeable with probability grow_axis per axial and grow_diag per
    diagonal permeable neighbour, until frac_perm of the lattice is
    permeable (the last sweep keeps a random subset of its new cells).
    The paper's own generators are not published; these are seeded
    stand-ins with its volume fractions."""
    rng = _rng(seed)
    lab = np.full((ny, nx), PORE, dtype=np.int8)
    yy, xx = np.mgrid[0:ny, 0:nx]
    target = frac_solid * nx * ny
    while np.count_nonzero(lab == IMPERMEABLE) < target:
        cx, cy = rng.uniform(0, nx), rng.uniform(0, ny)
        r = rng.uniform(*r_range)
        dx = (xx - cx + nx / 2) % nx - nx / 2
        dy = (yy - cy + ny / 2) % ny - ny / 2
        lab[dx * dx + dy * dy <= r * r] = IMPERMEABLE
    free = lab == PORE
    lab[free & (rng.uniform(size=lab.shape) < core_prob)] = PERMEABLE
    need = int(round(frac_perm * nx * ny))
    dirs = [((0, 1), grow_axis), ((0, -1), grow_axis), ((1, 0), grow_axis), ((-1, 0), grow_axis),
            ((1, 1), grow_diag), ((1, -1), grow_diag), ((-1, 1), grow_diag),
            ((-1, -1), grow_diag)]
    while True:
        perm = lab == PERMEABLE
        left = need - int(np.count_nonzero(perm))
        if left <= 0 or not np.any(lab == PORE):
            break
        new = np.zeros_like(perm)
        for (sy, sx), pr in dirs:
            nb = np.roll(perm, (sy, sx), axis=(0, 1))
            new |= nb & (lab == PORE) & (rng.uniform(size=lab.shape) < pr)
        cand = np.flatnonzero(new)
        if cand.size > left:
            cand = rng.choice(cand, left, replace=False)
        lab.flat[cand] = PERMEABLE
    return lab


def trimodal_medium(labels: np.ndarray, eps_ps: float, k_i_ps, kn_ps) -> Medium:
    """Fields of a labelled three-component medium: pores eps = 1, k = inf
    (no matrix), impermeable solids eps = 0 (k unused, set to 1), permeable
    solids eps_ps with the given k_i and Kn (scalars or [ny][nx] arrays
    read at the permeable cells)."""
    shp = labels.shape
    perm = labels == PERMEABLE
    eps = np.where(labels == PORE, 1.0, 0.0)
    eps[perm] = eps_ps
    k_i = np.where(labels == PORE, np.inf, 1.0)
    k_i[perm] = np.broadcast_to(np.asarray(k_i_ps, dtype=np.float64), shp)[perm]
    kn = np.zeros(shp)
    kn[perm] = np.broadcast_to(np.asarray(kn_ps, dtype=np.float64), shp)[perm]
    return Medium(eps, k_i, kn, "trimodal")
