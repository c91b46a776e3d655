"""Seeded synthetic galaxy catalogs shaped like the paper's workloads.

This module only generates inputs (positions and weights); it holds none of the
estimator's arithmetic. The paper measures on BOSS CMASS / MultiDark-Patchy
catalogs (Sec. 5.4) and on uniform periodic boxes (Sec. 5.1, 5.3); these
generators stand in for them:

* ``uniform_box``  -- Poisson points in a periodic cube (Sec. 5.1 test boxes).
* ``lognormal_box`` -- a log-normal density field: Gaussian field with power
  spectrum P(k) = A k^-1.5 exp(-(k/0.5)^2) on a mesh, variance normalised to
  sigma_G^2 = 1 in expectation, 1 + delta = exp(G) / <exp(G)>, then exactly N
  points drawn multinomially over cells with probability proportional to
  1 + delta and placed uniformly inside their cell.
* ``survey``       -- log-normal data cut to a non-periodic shell-and-cap mask
  (comoving radius 600-1400 Mpc/h, 60 degree cap about +z) plus uniform
  randoms in the same mask; ``survey_splits`` cuts the randoms into disjoint
  seeded splits (Sec. 4.2).
* ``lognormal_mesh`` -- the log-normal overdensity exp(G)/<exp(G)> - 1 itself on a
  periodic mesh (a gridded field, Sec. 3.2.2).

Positions are float32 in [0, L) for periodic boxes. All draws use numpy's
PCG64 with explicit seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np


def _wrap_f32(x: np.ndarray, box: float) -> np.ndarray:
    """Cast to float32 and fold any value that rounded up to L back into [0, L)."""
    xf = x.astype(np.float32)
    L = np.float32(box)
    xf[xf >= L] -= L
    xf[xf < 0] += L
    xf[xf >= L] = np.nextafter(L, np.float32(0))
    return xf


def uniform_box(n: int, box: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return _wrap_f32(rng.uniform(0.0, box, size=(n, 3)), box)


def gaussian_field(mesh: int, box: float, rng, slope: float = -1.5, kcut: float = 0.5,
                   sigma_g: float = 1.0) -> np.ndarray:
    """Real Gaussian field on a mesh^3 grid with P(k) propto k^slope exp(-(k/kcut)^2)."""
    noise = rng.standard_normal((mesh, mesh, mesh))
    nk = np.fft.rfftn(noise)
    kf = 2.0 * math.pi / box
    k1 = np.fft.fftfreq(mesh, d=1.0 / mesh) * kf
    kz = np.fft.rfftfreq(mesh, d=1.0 / mesh) * kf
    k2 = (k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
    k = np.sqrt(k2)
    with np.errstate(divide="ignore"):
        pk = np.where(k > 0, k ** slope * np.exp(-(k / kcut) ** 2), 0.0)
    # Full-grid sum of P over all modes (rfft half-plane weights: interior x2).
    wz = np.full(kz.shape, 2.0)
    wz[0] = 1.0
    if mesh % 2 == 0:
        wz[-1] = 1.0
    psum = float((pk * wz[None, None, :]).sum())
    # E|noise_k|^2 = mesh^3, so Var(G) = (c^2 / mesh^3) sum_k P(k); pick c for sigma_g.
    c2 = sigma_g ** 2 * mesh ** 3 / psum
    g = np.fft.irfftn(nk * np.sqrt(pk * c2), s=(mesh, mesh, mesh), axes=(0, 1, 2))
    return g


def lognormal_mesh(mesh: int, box: float, seed: int, **kw) -> np.ndarray:
    """Overdensity delta = exp(G) / <exp(G)> - 1 of the log-normal field on a periodic
    mesh^3 grid (float32, C order; read as [z][y][x] with x fastest)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eg = np.exp(gaussian_field(mesh, box, rng, **kw))
    return np.ascontiguousarray(eg / eg.mean() - 1.0, dtype=np.float32)


def _sample_cells(density: np.ndarray, n: int, rng) -> np.ndarray:
    p = density.ravel()
    p = p / p.sum()
    counts = rng.multinomial(n, p)
    return np.repeat(np.arange(p.size), counts)


def lognormal_box(n: int, box: float, mesh: int, seed: int, **kw) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    g = gaussian_field(mesh, box, rng, **kw)
    eg = np.exp(g)
    dens = eg / eg.mean()
    cells = _sample_cells(dens, n, rng)
    rng.shuffle(cells)
    iz = cells % mesh
    iy = (cells // mesh) % mesh
    ix = cells // (mesh * mesh)
    cell = box / mesh
    u = rng.uniform(0.0, 1.0, size=(n, 3))
    pos = np.stack([(ix + u[:, 0]) * cell, (iy + u[:, 1]) * cell, (iz + u[:, 2]) * cell], axis=1)
    return _wrap_f32(pos, box)


# survey mask: comoving radius [600, 1400] Mpc/h, cap of 60 degrees about +z
R_IN, R_OUT, COS_CAP = 600.0, 1400.0, 0.5


def in_mask(pos: np.ndarray) -> np.ndarray:
    r = np.sqrt((pos.astype(np.float64) ** 2).sum(axis=1))
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = pos[:, 2] / r
    return (r >= R_IN) & (r <= R_OUT) & (mu >= COS_CAP)


def survey_randoms(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.cbrt(rng.uniform(R_IN ** 3, R_OUT ** 3, size=n))
    mu = rng.uniform(COS_CAP, 1.0, size=n)
    phi = rng.uniform(0.0, 2 * math.pi, size=n)
    s = np.sqrt(1.0 - mu * mu)
    return np.stack([r * s * np.cos(phi), r * s * np.sin(phi), r * mu], axis=1).astype(np.float32)


def survey_data(n: int, seed: int, mesh: int = 256) -> np.ndarray:
    """Log-normal points inside the survey mask (field on a 2500 Mpc/h cube centred at z=1250)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = 2500.0
    origin = np.array([-1250.0, -1250.0, 0.0])
    g = gaussian_field(mesh, side, rng)
    eg = np.exp(g)
    dens = eg / eg.mean()
    cell = side / mesh
    out: List[np.ndarray] = []
    have = 0
    while have < n:
        cells = _sample_cells(dens, 4 * n, rng)
        iz = cells % mesh
        iy = (cells // mesh) % mesh
        ix = cells // (mesh * mesh)
        u = rng.uniform(0.0, 1.0, size=(len(cells), 3))
        pos = np.stack([(ix + u[:, 0]) * cell, (iy + u[:, 1]) * cell, (iz + u[:, 2]) * cell],
                       axis=1) + origin
        pos = pos[in_mask(pos)]
        rng.shuffle(pos)
        out.append(pos)
        have += len(pos)
    return np.concatenate(out)[:n].astype(np.float32)


@dataclass
class Workload:
    """One catalog plus the estimator settings it is measured with."""
    name: str
    pos: np.ndarray                 # float32 [n, 3]
    w: np.ndarray                   # float32 [n]
    edges: np.ndarray               # float64 [nr + 1]
    lmax: int
    orders: Sequence[int]
    box: float                      # > 0 periodic side, 0 non-periodic
    allparity: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.pos)


def linear_edges(rmin: float, rmax: float, nr: int) -> np.ndarray:
    return np.linspace(rmin, rmax, nr + 1)


def uniform4k_3pcf(n: int = 4096) -> Workload:
    """4,096 uniform points, periodic 250 Mpc/h cube, 10 shells 0-50, lmax 5, 3PCF."""
    pos = uniform_box(n, 250.0, seed=1001)
    return Workload("3pcf_uniform_4096_L250", pos, np.ones(n, np.float32),
                    linear_edges(0.0, 50.0, 10), 5, (3,), 250.0)


def paper_uniform_1500(n: int = 50_000, lmax: int = 5, orders=(3, 4)) -> Workload:
    """The paper's timing catalog (Table 2): about 5e4 uniform points in a periodic
    1500 Mpc/h box, pairs up to r_max = 200 Mpc/h in 10 shells (r_min = 0)."""
    pos = uniform_box(n, 1500.0, seed=1500)
    return Workload("uniform_%dk_L1500" % (n // 1000), pos, np.ones(n, np.float32),
                    linear_edges(0.0, 200.0, 10), lmax, tuple(orders), 1500.0)


def lognormal200k_4pcf(n: int = 200_000, mesh: int = 256) -> Workload:
    """200k log-normal points, periodic 1000 Mpc/h cube, 10 shells 20-160, lmax 5, 3+4PCF."""
    pos = lognormal_box(n, 1000.0, mesh, seed=1002)
    return Workload("4pcf3pcf_lognormal_200k_L1000", pos, np.ones(n, np.float32),
                    linear_edges(20.0, 160.0, 10), 5, (3, 4), 1000.0)


def lognormal100k_5pcf(n: int = 100_000, mesh: int = 256) -> Workload:
    """100k log-normal points, periodic 1000 Mpc/h cube, 8 shells 20-160, lmax 4, 5PCF."""
    pos = lognormal_box(n, 1000.0, mesh, seed=1004)
    return Workload("5pcf_lognormal_100k_L1000", pos, np.ones(n, np.float32),
                    linear_edges(20.0, 160.0, 8), 4, (5,), 1000.0)


def survey_dmr_and_randoms(n_data: int = 400_000, n_rand: int = 1_600_000, mesh: int = 256):
    """D-R catalog (data +1, randoms -N_D/N_R) and the R-only catalog (randoms +N_D/N_R)."""
    d = survey_data(n_data, seed=1003, mesh=mesh)
    r = survey_randoms(n_rand, seed=2003)
    ratio = n_data / n_rand
    pos = np.concatenate([d, r])
    w = np.concatenate([np.ones(n_data, np.float32), np.full(n_rand, -ratio, np.float32)])
    edges = linear_edges(20.0, 160.0, 10)
    dr = Workload("survey_DmR_%dk_%dk" % (n_data // 1000, n_rand // 1000), pos, w, edges, 5,
                  (3, 4), 0.0)
    rr = Workload("survey_R_%dk" % (n_rand // 1000), r, np.full(n_rand, ratio, np.float32),
                  edges, 5, (3, 4), 0.0)
    return dr, rr


def survey_splits(n_data: int = 400_000, n_rand: int = 1_600_000, nsplit: int = 4, mesh: int = 256):
    """Survey data (weight +1) and its randoms cut into nsplit disjoint seeded splits, split k
    weighted -N_D / N_k (Sec. 4.2: random splits co-added)."""
    d = survey_data(n_data, seed=1003, mesh=mesh)
    r = survey_randoms(n_rand, seed=2003)
    rng = np.random.Generator(np.random.PCG64(4003))
    parts = np.array_split(rng.permutation(n_rand), nsplit)
    splits = [(r[np.sort(p)], np.full(len(p), -n_data / len(p), np.float32)) for p in parts]
    return d, np.ones(n_data, np.float32), splits, linear_edges(20.0, 160.0, 10)


def lognormal_6pcf(n: int = 50_000, mesh: int = 128) -> Workload:
    """50k log-normal points, periodic 1000 Mpc/h cube, 8 shells 20-160, lmax 2, 6PCF."""
    pos = lognormal_box(n, 1000.0, mesh, seed=1006)
    return Workload("6pcf_lognormal_%dk_L1000" % (n // 1000), pos, np.ones(n, np.float32),
                    linear_edges(20.0, 160.0, 8), 2, (6,), 1000.0)


def survey_subset(dr: "Workload", rr: "Workload", n_data: int = 4000, n_rand: int = 16000,
              seed: int = 3003):
    """Seeded subset of the survey catalogs (n_data data points, n_rand randoms), with the
    randoms re-weighted to -n_data/n_rand (D-R) and +n_data/n_rand (R only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nd = int(np.sum(dr.w > 0))
    di = np.sort(rng.choice(nd, n_data, replace=False))
    ri = np.sort(rng.choice(len(rr.pos), n_rand, replace=False))
    ratio = n_data / n_rand
    pos = np.concatenate([dr.pos[di], rr.pos[ri]])
    w = np.concatenate([np.ones(n_data, np.float32), np.full(n_rand, -ratio, np.float32)])
    sub_dr = Workload(dr.name + "_subset%dk" % ((n_data + n_rand) // 1000), pos, w, dr.edges, dr.lmax,
                      dr.orders, 0.0)
    sub_rr = Workload(rr.name + "_subset%dk" % (n_rand // 1000), rr.pos[ri],
                      np.full(n_rand, ratio, np.float32), rr.edges, rr.lmax, rr.orders, 0.0)
    return sub_dr, sub_rr


def batch64_sizes(ncat: int = 64) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(5000))
    return np.round(np.exp(rng.uniform(math.log(2e4), math.log(3e5), size=ncat))).astype(np.int64)


def batch64_lognormal(ncat: int = 64, mesh: int = 128, sizes: Optional[np.ndarray] = None):
    """64 log-normal periodic catalogs with sizes log-uniform in [2e4, 3e5]."""
    if sizes is None:
        sizes = batch64_sizes(ncat)
    cats = [lognormal_box(int(s), 1000.0, mesh, seed=5000 + k) for k, s in enumerate(sizes)]
    return cats, linear_edges(20.0, 160.0, 10)
