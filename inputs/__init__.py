"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method itself (no energy, gradient,
Hessian, eigensolver, ascent or charge).  It only draws reproducible random
numbers and lays out initial spin textures on the periodic triangular lattice,
so that both sides of every parity test start from bit-identical inputs.

Random numbers
--------------
* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) used in counter mode: draw ``k`` of stream
  ``seed`` is ``mix(seed + (k + 1) * 0x9E3779B97F4A7C15)``, which is exactly the
  k-th output of the sequential generator started at state ``seed``.
* Uniforms in [0, 1): the top 53 bits of a draw times 2**-53.
* Normals: Box & Muller (1958), one pair of normals per pair of uniforms.

Textures (the paper does not state how its initial states were seeded)
--------------------------------------------------------------------
* Skyrmion of radius R centred at c (minimum-image distance on the periodic
  rhombus): theta(r) = 2 atan2(sinh(R/w), sinh(r/w)), w = 2, so the core points
  down (-z) in a +z background; m = (sin th cos(phi+gamma), sin th sin(phi+gamma),
  cos th).  Antiskyrmion: phi -> -phi.  Meron: theta clipped to at least pi/2
  inside the disk r <= 2R.  Biskyrmion: two skyrmions 2.5 R apart.
* Gaussian noise N(0, sigma) per component, then each spin is rescaled to unit
  length.

Lattice layout: arrays are ``(3, L2, L1)`` float64, component-major (SoA), site
(i1, i2) at position i1*a1 + i2*a2 with a1 = (1, 0), a2 = (1/2, sqrt(3)/2).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Model parameters of the five synthetic workloads (meV; field mu*B along +z).
WORKLOADS = {
    1: dict(name="plain-fp64-32x32", L1=32, L2=32, J=(1.0,), D=0.3, K=0.05, muB=0.02),
    2: dict(name="fp32-vs-fp64-256x256", L1=256, L2=256, J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02),
    3: dict(name="batched-128x128", L1=128, L2=128, J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02),
    4: dict(name="roofline-2048x2048", L1=2048, L2=2048, J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02),
    5: dict(name="autograd-512x512", L1=512, L2=512, J=(1.0, -0.1, -0.05), D=0.3, K=0.05, muB=0.02),
}


def workload_seed(config: int, walker: int) -> int:
    """Seed of walker ``walker`` in workload ``config``: 1000*config + walker."""
    return 1000 * int(config) + int(walker)


# ----------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------
def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream started at ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` uniforms in [0, 1) from the top 53 bits of SplitMix64 draws."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` standard normals by Box-Muller over consecutive uniform pairs."""
    npair = (n + 1) // 2
    u = uniform(seed, 2 * npair, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]: log is finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:n]


def gaussian_field(seed: int, L1: int, L2: int, offset: int = 0) -> np.ndarray:
    """A (3, L2, L1) array of independent standard normals."""
    return normal(seed, 3 * L1 * L2, offset).reshape(3, L2, L1)


# ----------------------------------------------------------------------------
# geometry (positions only)
# ----------------------------------------------------------------------------
SQRT3_2 = math.sqrt(3.0) / 2.0


def min_image(L1: int, L2: int, c1: float, c2: float):
    """Cartesian displacement (dx, dy) of every site from centre (c1, c2), both in
    lattice-index coordinates, taking the shortest periodic image."""
    i2, i1 = np.meshgrid(np.arange(L2, dtype=np.float64), np.arange(L1, dtype=np.float64), indexing="ij")
    d1 = np.mod(i1 - c1 + 0.5 * L1, L1) - 0.5 * L1
    d2 = np.mod(i2 - c2 + 0.5 * L2, L2) - 0.5 * L2
    best_dx = best_dy = None
    best_r2 = None
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            e1 = d1 + a * L1
            e2 = d2 + b * L2
            dx = e1 + 0.5 * e2
            dy = SQRT3_2 * e2
            r2 = dx * dx + dy * dy
            if best_r2 is None:
                best_dx, best_dy, best_r2 = dx, dy, r2
            else:
                take = r2 < best_r2
                best_dx = np.where(take, dx, best_dx)
                best_dy = np.where(take, dy, best_dy)
                best_r2 = np.where(take, r2, best_r2)
    return best_dx, best_dy


# ----------------------------------------------------------------------------
# textures
# ----------------------------------------------------------------------------
def ferromagnet(L1: int, L2: int) -> np.ndarray:
    m = np.zeros((3, L2, L1))
    m[2] = 1.0
    return m


def _theta_profile(r, R, w=2.0):
    return 2.0 * np.arctan2(np.sinh(R / w), np.sinh(r / w))


def _texture(L1, L2, c1, c2, R, helicity, vorticity, meron=False):
    dx, dy = min_image(L1, L2, c1, c2)
    r = np.hypot(dx, dy)
    phi = vorticity * np.arctan2(dy, dx)
    th = _theta_profile(r, R)
    if meron:
        th = np.where(r <= 2.0 * R, np.maximum(th, 0.5 * math.pi), th)
    return th, phi + helicity, r


def _compose(L1, L2, parts):
    """Superpose localised textures on a +z background: each part supplies
    (theta, azimuth); where textures overlap the one with the larger polar
    angle (deeper core) wins."""
    th_all = np.zeros((L2, L1))
    az_all = np.zeros((L2, L1))
    for th, az in parts:
        take = th > th_all
        th_all = np.where(take, th, th_all)
        az_all = np.where(take, az, az_all)
    m = np.empty((3, L2, L1))
    m[0] = np.sin(th_all) * np.cos(az_all)
    m[1] = np.sin(th_all) * np.sin(az_all)
    m[2] = np.cos(th_all)
    return m


def skyrmion(L1, L2, R, c=None, helicity=math.pi, anti=False):
    """Isolated (anti)skyrmion of radius R (sites) at centre c (index coords)."""
    if c is None:
        c = (0.5 * (L1 - 1), 0.5 * (L2 - 1))
    th, az, _ = _texture(L1, L2, c[0], c[1], R, helicity, -1.0 if anti else 1.0)
    return _compose(L1, L2, [(th, az)])


def meron(L1, L2, R, c=None, helicity=math.pi):
    if c is None:
        c = (0.5 * (L1 - 1), 0.5 * (L2 - 1))
    th, az, _ = _texture(L1, L2, c[0], c[1], R, helicity, 1.0, meron=True)
    return _compose(L1, L2, [(th, az)])


def biskyrmion(L1, L2, R, c=None, helicity=math.pi):
    """Two skyrmions (total charge 2) whose centres are 2.5 R apart along a1."""
    if c is None:
        c = (0.5 * (L1 - 1), 0.5 * (L2 - 1))
    sep = 2.5 * R
    parts = []
    for s in (-0.5, 0.5):
        th, az, _ = _texture(L1, L2, c[0] + s * sep, c[1], R, helicity, 1.0)
        parts.append((th, az))
    return _compose(L1, L2, parts)


def multi_texture(L1, L2, charge: int, R: float, seed: int, helicity=math.pi):
    """|charge| skyrmions (charge > 0) or antiskyrmions (charge < 0) at seeded,
    non-overlapping centres; charge 0 gives a skyrmion-antiskyrmion pair."""
    if charge == 0:
        kinds = [1.0, -1.0]
    else:
        kinds = [1.0 if charge > 0 else -1.0] * abs(charge)
    centres = []
    u = uniform(seed, 400, offset=0)
    k = 0
    min_sep = 3.0 * R
    while len(centres) < len(kinds) and k + 1 < len(u):
        c = (u[k] * L1, u[k + 1] * L2)
        k += 2
        ok = True
        for cc in centres:
            dx, dy = min_image(L1, L2, cc[0], cc[1])
            j1 = int(round(c[0])) % L1
            j2 = int(round(c[1])) % L2
            if math.hypot(dx[j2, j1], dy[j2, j1]) < min_sep:
                ok = False
                break
        if ok:
            centres.append(c)
    if len(centres) < len(kinds):
        raise ValueError("lattice too small for the requested texture")
    parts = []
    for kind, c in zip(kinds, centres):
        th, az, _ = _texture(L1, L2, c[0], c[1], R, helicity, kind)
        parts.append((th, az))
    return _compose(L1, L2, parts)


def add_noise(m: np.ndarray, sigma: float, seed: int, mask: np.ndarray | None = None, offset: int = 0) -> np.ndarray:
    """m + N(0, sigma) per component (optionally only where ``mask``), then each
    spin rescaled to unit length."""
    L2, L1 = m.shape[1:]
    noise = sigma * gaussian_field(seed, L1, L2, offset)
    if mask is not None:
        noise = noise * mask[None]
    out = m + noise
    out /= np.sqrt(np.sum(out * out, axis=0))[None]
    return out


def disk_mask(L1, L2, c, radius):
    dx, dy = min_image(L1, L2, c[0], c[1])
    return (np.hypot(dx, dy) <= radius).astype(np.float64)


# ----------------------------------------------------------------------------
# the five workloads' initial states
# ----------------------------------------------------------------------------
def workload1_state():
    """32x32, skyrmion R=4 at the centre, N(0, 0.01) noise, seed 1000."""
    p = WORKLOADS[1]
    m = skyrmion(p["L1"], p["L2"], 4.0)
    return add_noise(m, 0.01, workload_seed(1, 0))


def workload2_states(n=20):
    """256x256: 7 skyrmions, 7 antiskyrmions, 6 merons; R ~ U[4, 8], seeded
    random centres; seed 2000 + w."""
    p = WORKLOADS[2]
    out = []
    for w in range(n):
        s = workload_seed(2, w)
        u = uniform(s, 3)
        R = 4.0 + 4.0 * u[0]
        c = (u[1] * p["L1"], u[2] * p["L2"])
        kind = w % 20
        if kind < 7:
            m = skyrmion(p["L1"], p["L2"], R, c)
        elif kind < 14:
            m = skyrmion(p["L1"], p["L2"], R, c, anti=True)
        else:
            m = meron(p["L1"], p["L2"], R, c)
        out.append(add_noise(m, 0.01, s, offset=8))
    return out


def workload3_walker(w: int, L1: int = 128, L2: int | None = None):
    """Batched-explorer walker w: random charge in {-2..2}, R ~ U[3, 5], masked
    N(0, 0.05) perturbation inside a disk of radius 2R (x = x0 + P_Omega delta)."""
    if L2 is None:
        L2 = L1
    s = workload_seed(3, w)
    u = uniform(s, 4)
    q = int(math.floor(u[0] * 5.0)) - 2
    R = 3.0 + 2.0 * u[1]
    m = multi_texture(L1, L2, q, R, s + 7919)
    c = (u[2] * L1, u[3] * L2)
    mask = disk_mask(L1, L2, c, 2.0 * R)
    return add_noise(m, 0.05, s, mask=mask, offset=16)


def workload3_mixed_sides(n=64):
    """Side lengths of the mixed batch, uniform in {48..192}."""
    u = uniform(workload_seed(3, 999), n)
    return [48 + int(math.floor(x * 145.0)) for x in u]


def workload4_state():
    """2048x2048 biskyrmion (Q = 2), R = 8, N(0, 0.01) noise, seed 4000."""
    p = WORKLOADS[4]
    m = biskyrmion(p["L1"], p["L2"], 8.0)
    return add_noise(m, 0.01, workload_seed(4, 0))


def workload5_state():
    p = WORKLOADS[5]
    m = biskyrmion(p["L1"], p["L2"], 8.0)
    return add_noise(m, 0.05, workload_seed(5, 0))


def random_pairs(seed: int, reach: int, n_offsets: int):
    """A pair list for the general pair-list Hamiltonian: up to n_offsets
    distinct offsets (d1, d2) with |d1|, |d2| <= reach, each listed with its
    negative; J ~ 0.3 N(0,1), D ~ 0.2 N(0,1)^3 for the first and (J, -D) for
    the negative, so the list has the closure an ordered-pair sum needs."""
    vals = normal(seed, 8 * n_offsets).reshape(n_offsets, 8)
    seen, out = set(), []
    for k in range(n_offsets):
        d1 = int(round(vals[k, 0] * 10)) % (2 * reach + 1) - reach
        d2 = int(round(vals[k, 1] * 10)) % (2 * reach + 1) - reach
        if (d1, d2) == (0, 0) or (d1, d2) in seen or (-d1, -d2) in seen:
            continue
        seen.add((d1, d2))
        J = 0.3 * float(vals[k, 2])
        D = tuple(0.2 * float(x) for x in vals[k, 3:6])
        out.append((d1, d2, J, D))
        out.append((-d1, -d2, J, tuple(-x for x in D)))
    return out


# ----------------------------------------------------------------------------
# Pd/Fe/Ir(111) pair list from the paper's printed parameter tables
# ----------------------------------------------------------------------------
MRY_TO_MEV = 13.605693122994  # 1 mRy in meV (Rydberg energy 13.605693122994 eV)


def pdfeir_table():
    """The 360 printed rows of Supplementary Note 4 (exchange and DMI tables,
    same pair order): array of [J, Dx, Dy, Dz, |r|] in mRy and the printed
    length unit (nearest neighbours at 0.707107)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pdfeir_supp_note4.txt")
    return np.loadtxt(path, comments="#")


def _shell_offsets(n2: int, reach: int):
    """Index-space offsets (d1, d2) with d1^2 + d1 d2 + d2^2 = n2 (squared
    length in nearest-neighbour units on the triangular lattice)."""
    return [(d1, d2) for d1 in range(-reach, reach + 1) for d2 in range(-reach, reach + 1)
            if d1 * d1 + d1 * d2 + d2 * d2 == n2]


def pdfeir_assignment(reach: int = 12):
    """The row-to-offset assignment of reading R23 (see pdfeir_pairs): a list
    of (row, d1, d2, Dx, Dy) with the in-plane DMI components of the row in the
    rotated frame (mRy)."""
    tab = pdfeir_table()
    rnn = 0.7071067811865476
    n2 = np.rint((tab[:, 4] / rnn) ** 2).astype(int)
    # frame: the nearest-neighbour D vectors' in-plane angles minus 90 degrees
    # are the bond angles; rotate them onto multiples of 60 degrees
    nn = tab[n2 == 1]
    bond = np.arctan2(nn[:, 2], nn[:, 1]) - 0.5 * math.pi
    rot = -np.angle(np.exp(6j * bond).mean()) / 6.0
    c, s = math.cos(rot), math.sin(rot)
    out = []
    for sh in sorted(set(n2.tolist())):
        rows = np.nonzero(n2 == sh)[0]
        offs = _shell_offsets(int(sh), reach)
        if len(offs) != len(rows):
            raise ValueError(f"shell {sh}: {len(rows)} rows for {len(offs)} offsets")
        Dx = c * tab[rows, 1] - s * tab[rows, 2]
        Dy = s * tab[rows, 1] + c * tab[rows, 2]
        ang_rows = np.arctan2(Dy, Dx)
        # z x r_hat for r = d1 a1 + d2 a2 (a1 = (1, 0), a2 = (1/2, sqrt(3)/2))
        ang_offs = np.array([math.atan2(d1 + 0.5 * d2, -(math.sqrt(3) / 2) * d2) for d1, d2 in offs])
        ir = np.argsort(ang_rows, kind="stable")
        io = np.argsort(ang_offs, kind="stable")
        best, best_shift = None, 0
        for sft in range(len(rows)):
            dif = np.angle(np.exp(1j * (ang_rows[ir] - ang_offs[np.roll(io, -sft)])))
            cost = float(np.sum(dif * dif))
            if best is None or cost < best - 1e-12:
                best, best_shift = cost, sft
        io = np.roll(io, -best_shift)
        for a, b in zip(ir, io):
            out.append((int(rows[a]), offs[b][0], offs[b][1], float(Dx[a]), float(Dy[a])))
    return out


def pdfeir_pairs(reach: int = 12):
    """Pair list (d1, d2, J, (Dx, Dy, Dz)) in meV for the general pair-list
    Hamiltonian, from the printed tables (reading R23):

    * |r| in units of the printed nearest-neighbour distance (0.707107) gives
      the shell n2 = |r|^2, whose triangular-lattice offsets the table's rows
      of that length populate (the row counts equal the shell sizes).
    * The tables give no bond directions.  The frame is rotated about z so that
      the nearest-neighbour DMI vectors are Neel, D = |D| z x r_hat, with the
      bonds along a1 and its 60-degree images; in every shell the rows, sorted
      by the angle of the in-plane part of D, are matched in that cyclic order
      to the offsets sorted by the angle of z x r_hat, with the cyclic shift of
      least angular mismatch.  Each row's J goes with its D (one pair order).
    * Of the two rows of a bond (d and -d) the one on the half plane d1 > 0 or
      (d1 == 0, d2 > 0) is kept and its reverse is set to (J, -D), which is the
      closure an ordered-pair sum needs.
    * mRy -> meV by the Rydberg energy."""
    tab = pdfeir_table()
    out = {}
    for row, d1, d2, Dx, Dy in pdfeir_assignment(reach):
        if d1 > 0 or (d1 == 0 and d2 > 0):
            out[(d1, d2)] = (float(tab[row, 0]) * MRY_TO_MEV,
                             (Dx * MRY_TO_MEV, Dy * MRY_TO_MEV, float(tab[row, 3]) * MRY_TO_MEV))
    pairs = []
    for (d1, d2), (J, D) in sorted(out.items()):
        pairs.append((d1, d2, J, D))
        pairs.append((-d1, -d2, J, (-D[0], -D[1], -D[2])))
    return pairs
