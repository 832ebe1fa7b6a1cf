"""Seeded synthetic inputs for the Cr-film / carbon-indenter nano-indentation MD.

This module builds the initial state that both the CUDA path and the CPU oracle
receive: lattice positions, the rigid indenter, the fixed-atom mask, the
velocities and the per-workload options.  It holds none of the method's
arithmetic (no potential, neighbour list, force or integrator); it only lays
atoms on lattices and draws random numbers, so the two implementations can be
fed the *same arrays* and never depend on matching random generators.

Film (Sec. 2.5, "System initialization and loading"): a BCC Cr film of
nx x ny x nz unit cells.  The default form is periodic in x and y
(2 * nx * ny * nz atoms); the paper-literal form has free lateral faces and
(nx+1)(ny+1)(nz+1) + nx*ny*nz atoms (2331 atoms for 10^3 cells, 11054 for
19x19x14, 100111 for 40x40x30, 132921 for 40^3, Sec. 2.5 and Sec. 4).

Indenter (Sec. 2.5 and the Appendix): a rigid hemisphere of diamond-lattice
carbon, cubic axes parallel to the film, sphere centred on a lattice atom,
boundary-inclusive (|p| <= R), lower half (p_z <= 0), centred laterally, its
lowest atom `gap` above the top Cr plane.

Velocities (Sec. 2.5): each component ~ N(0, k_B T / m) for mobile atoms,
then the centre-of-mass velocity of the mobile atoms is removed; fixed atoms
have v = 0.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Units: Angstrom, eV, fs, u.
A_CR = 2.885            # BCC Cr lattice constant (Angstrom)
A_DIAMOND = 3.567       # diamond-C lattice constant (Angstrom)
MASS_CR = 51.9961       # standard atomic weight of Cr (u); the paper does not print it
KB_EV = 8.617333262e-5  # Boltzmann constant (eV/K)
EV_PER_U_A2_FS2 = 1.0 / 9.6485332e-3  # 1 u*A^2/fs^2 in eV
MS_TO_A_FS = 1e-5       # 1 m/s in Angstrom/fs

_DIAMOND_BASIS = np.array(
    [[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
     [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])


def bcc_film(nx: int, ny: int, nz: int, a: float = A_CR, free_lateral: bool = False):
    """BCC film positions, (N, 3) float64, sorted by (z, y, x).

    Periodic form: corner sites (i, j, k) a and body centres (i+1/2, j+1/2, k+1/2) a
    for 0 <= i < nx, 0 <= j < ny, 0 <= k < nz; the lateral box is [0, nx a) x [0, ny a).
    Free-lateral (paper-literal) form: corners for 0 <= i <= nx etc. plus the
    nx*ny*nz body centres.
    """
    if free_lateral:
        ci = np.arange(nx + 1); cj = np.arange(ny + 1); ck = np.arange(nz + 1)
    else:
        ci = np.arange(nx); cj = np.arange(ny); ck = np.arange(nz)
    K, J, I = np.meshgrid(ck, cj, ci, indexing="ij")
    corners = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    centres = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64) + 0.5
    pos = np.concatenate([corners, centres]) * a
    order = np.lexsort((pos[:, 0], pos[:, 1], pos[:, 2]))
    return np.ascontiguousarray(pos[order])


def bcc_count(nx: int, ny: int, nz: int, free_lateral: bool) -> int:
    """Closed-form atom count of `bcc_film`."""
    if free_lateral:
        return (nx + 1) * (ny + 1) * (nz + 1) + nx * ny * nz
    return 2 * nx * ny * nz


def fixed_planes_mask(pos: np.ndarray, a: float, n_planes: int) -> np.ndarray:
    """1 for atoms in the bottom `n_planes` atomic (001) planes (spacing a/2), else 0.

    Two planes make the paper's "bottom-most layer of unit cells" (Sec. 2.5).
    """
    zmin = pos[:, 2].min()
    return ((pos[:, 2] - zmin) < (n_planes - 0.5) * 0.5 * a).astype(np.uint8)


def diamond_hemisphere(R: float, a: float = A_DIAMOND) -> np.ndarray:
    """Lower half-ball of a diamond lattice, relative to the sphere centre (an atom)."""
    m = int(math.ceil(R / a)) + 2
    g = np.arange(-m, m + 1)
    I, J, K = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([I.ravel(), J.ravel(), K.ravel()], 1).astype(np.float64)
    p = ((cells[:, None, :] + _DIAMOND_BASIS[None]) * a).reshape(-1, 3)
    r = np.sqrt((p * p).sum(1))
    sel = (r <= R + 1e-9) & (p[:, 2] <= 1e-9)
    p = p[sel]
    order = np.lexsort((p[:, 0], p[:, 1], p[:, 2]))
    return np.ascontiguousarray(p[order])


def maxwell_velocities(n: int, T: float, mass: float, fixed: np.ndarray,
                       rng: np.random.Generator) -> np.ndarray:
    """Gaussian velocities (Angstrom/fs) at temperature T, COM of mobile atoms removed."""
    sigma = math.sqrt(KB_EV * T / mass / EV_PER_U_A2_FS2) if T > 0 else 0.0
    v = rng.standard_normal((n, 3)) * sigma
    mob = fixed == 0
    v[~mob] = 0.0
    if mob.any():
        v[mob] -= v[mob].mean(0)
    return np.ascontiguousarray(v)


@dataclasses.dataclass
class Replica:
    """One independent indentation system (all arrays float64 C-contiguous, AoS x,y,z)."""
    name: str
    x_cr: np.ndarray          # (n_cr, 3) positions
    v_cr: np.ndarray          # (n_cr, 3) velocities, Angstrom/fs
    fixed: np.ndarray         # (n_cr,) uint8
    x_c: np.ndarray           # (n_c, 3) indenter atoms at t = 0
    box_lo: np.ndarray        # (3,)
    box_hi: np.ndarray        # (3,)
    periodic: np.ndarray      # (3,) int32
    z_indenter0: float        # indenter displacement at t = 0 (Angstrom)
    v_indenter: float         # indenter displacement rate (Angstrom/fs), negative = downwards
    dt: float                 # fs
    mass_cr: float            # u
    temperature: float        # K (the draw only)
    z_surface0: float         # top Cr plane at t = 0

    @property
    def n_cr(self) -> int:
        return int(self.x_cr.shape[0])

    @property
    def n_c(self) -> int:
        return int(self.x_c.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    replicas: List[Replica]
    steps: int
    skin: float = 0.3
    rebuild_every: int = 0
    precision: str = "mixed"

    @property
    def n_cr(self) -> int:
        return sum(r.n_cr for r in self.replicas)

    @property
    def n_c(self) -> int:
        return sum(r.n_c for r in self.replicas)


def make_replica(name: str, nx: int, ny: int, nz: int, R: float, T: float, seed: int,
                 n_fixed_planes: int = 2, gap: float = 3.0, v_ind_ms: float = 20.0,
                 dt: float = 1.0, free_lateral: bool = False, periodic_z: bool = False,
                 z_pad: float = 12.0) -> Replica:
    """Film + indenter + velocities for one system.

    The cell-grid domain in a non-periodic direction spans the film with `z_pad`
    Angstrom of room on each side (an atom that leaves it is reported as lost).
    """
    rng = np.random.default_rng(seed)
    x = bcc_film(nx, ny, nz, A_CR, free_lateral)
    fixed = fixed_planes_mask(x, A_CR, n_fixed_planes) if n_fixed_planes > 0 else np.zeros(len(x), np.uint8)
    v = maxwell_velocities(len(x), T, MASS_CR, fixed, rng)
    lo = np.zeros(3); hi = np.zeros(3)
    per = np.array([0, 0, 1 if periodic_z else 0], np.int32)
    if free_lateral:
        lo[:2] = -z_pad; hi[0] = nx * A_CR + z_pad; hi[1] = ny * A_CR + z_pad
    else:
        per[:2] = 1; hi[0] = nx * A_CR; hi[1] = ny * A_CR
    if periodic_z:
        lo[2] = 0.0; hi[2] = nz * A_CR
    else:
        lo[2] = x[:, 2].min() - z_pad; hi[2] = x[:, 2].max() + z_pad
    z_top = float(x[:, 2].max())
    if R > 0:
        c = diamond_hemisphere(R)
        cx = 0.5 * (nx * A_CR) if not free_lateral else 0.5 * nx * A_CR
        cy = 0.5 * (ny * A_CR) if not free_lateral else 0.5 * ny * A_CR
        c = c + np.array([cx, cy, z_top + gap - c[:, 2].min()])
    else:
        c = np.zeros((0, 3))
    return Replica(name=name, x_cr=x, v_cr=v, fixed=fixed, x_c=np.ascontiguousarray(c),
                   box_lo=lo, box_hi=hi, periodic=per, z_indenter0=0.0,
                   v_indenter=-v_ind_ms * MS_TO_A_FS, dt=dt, mass_cr=MASS_CR,
                   temperature=T, z_surface0=z_top)


RC_MORSE_DEFAULT = 6.0


def batched_replicas(n: int = 256, seed_base: int = 1507 * 1000, rc_morse: float = RC_MORSE_DEFAULT,
                     dt: float = 1.0) -> List[Replica]:
    """Uneven replicas: n_xy ~ U{6..24} (square films), n_z ~ U{6..12}, R ~ U(5, 15) A,
    T ~ U(100, 500) K; n_xy redrawn until L_xy >= 2 R + 2 rc_morse so the minimum
    image stays valid for the Cr-C pairs."""
    out = []
    for r in range(n):
        rng = np.random.default_rng(seed_base + r)
        R = float(rng.uniform(5.0, 15.0))
        T = float(rng.uniform(100.0, 500.0))
        nz = int(rng.integers(6, 13))
        while True:
            nxy = int(rng.integers(6, 25))
            if nxy * A_CR >= 2 * R + 2 * rc_morse:
                break
        out.append(make_replica(f"replica{r}", nxy, nxy, nz, R, T, seed=int(rng.integers(1 << 31)),
                                n_fixed_planes=2, dt=dt))
    return out


# Workload presets (seed = 1507 + preset index).
PRESETS = {
    # name: (nx, ny, nz, R, fixed planes, steps)
    "tiny": (8, 8, 8, 6.0, 2, 100),
    "64k": (40, 40, 20, 15.0, 3, 2000),
    "1M": (100, 100, 50, 30.0, 2, 1000),
    "8M": (200, 200, 100, 60.0, 2, 500),
}
_PRESET_INDEX = {"tiny": 0, "64k": 1, "1M": 2, "8M": 3, "batched": 4}


def make_workload(name: str, T: float = 300.0, n_replicas: int = 256,
                  precision: Optional[str] = None) -> Workload:
    """Build one of the preset workloads ('tiny', '64k', '1M', '8M', 'batched')."""
    if name == "batched":
        reps = batched_replicas(n_replicas)
        return Workload("batched", reps, steps=1000, precision=precision or "mixed")
    nx, ny, nz, R, nf, steps = PRESETS[name]
    rep = make_replica(name, nx, ny, nz, R, T, seed=1507 + _PRESET_INDEX[name], n_fixed_planes=nf)
    prec = precision or ("fp64" if name == "tiny" else "mixed")
    return Workload(name, [rep], steps=steps, precision=prec)


def paper_cube(n: int, T: float = 300.0, seed: int = 1507) -> Replica:
    """The paper's timing workload (Table 2, Sec. 4): a cube of n^3 BCC unit cells with free
    lateral faces, (n+1)^3 + n^3 atoms (2331 / 17261 / 132921 for n = 10 / 20 / 40), two
    fixed bottom planes, the indenter disabled."""
    return make_replica(f"cube{n}", n, n, n, 0.0, T, seed=seed + n, n_fixed_planes=2, free_lateral=True)


def small_cluster(n_side: int = 3, a: float = A_CR, jitter: float = 0.05, seed: int = 7,
                  vacuum: float = 10.0) -> Replica:
    """A small free BCC cluster with random displacements (no periodicity, no indenter)."""
    rng = np.random.default_rng(seed)
    x = bcc_film(n_side, n_side, n_side, a, free_lateral=True)
    x = x + rng.uniform(-jitter, jitter, x.shape)
    lo = x.min(0) - vacuum; hi = x.max(0) + vacuum
    return Replica(name="cluster", x_cr=np.ascontiguousarray(x), v_cr=np.zeros_like(x),
                   fixed=np.zeros(len(x), np.uint8), x_c=np.zeros((0, 3)), box_lo=lo, box_hi=hi,
                   periodic=np.zeros(3, np.int32), z_indenter0=0.0, v_indenter=0.0, dt=1.0,
                   mass_cr=MASS_CR, temperature=0.0, z_surface0=float(x[:, 2].max()))


def paper_indentation_film(T: float = 10.0, seed: int = 1507 + 5) -> Replica:
    """The paper's nano-indentation system (Sec. 2.5, Sec. 4.3): a Cr film of 19 x 19 x 14 BCC
    unit cells with free lateral faces (11054 atoms), the bottom layer of unit cells (two
    atomic planes) fixed, velocities at 10 K, and a diamond hemisphere of radius 9.78 A
    (the paper's 394 C; the lattice registration is not printed) 3 A above the top plane,
    moving at 10 m/s."""
    return make_replica("p11k", 19, 19, 14, 9.78, T, seed=seed, n_fixed_planes=2, gap=3.0,
                        v_ind_ms=10.0, free_lateral=True)
