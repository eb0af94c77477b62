"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module only draws random numbers and lays out spacetree refinement flags.
It contains none of the particle-in-cell arithmetic (no binning, deposit,
solve, gather or push): both the CUDA path and the CPU oracle receive the
arrays produced here and nothing else.

Conventions (the paper leaves them open; the same ones are used everywhere):

* Domain: the periodic unit square/cube [0,1)^d, k = 3 spacetree (Section 4).
* A tree is given as level-order (breadth-first) refinement flags: entry i is 1
  when node i is refined.  The root is node 0; the 3^d children of a refined
  node are appended in local-digit order l = i0 + 3*i1 + 9*i2 (x fastest).
* Particles are structure-of-arrays: ``x[a][p]``, ``v[a][p]`` for axis a.
* Plasma units: omega_p = 1, eps0 = 1, electron charge per particle -1/N,
  mass 1/N (q/m = -1), immobile ion background of density +1 (Appendix A).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from statistics import NormalDist

__all__ = [
    "uniform_tree_flags",
    "tree_flags_from_predicate",
    "Workload",
    "langmuir",
    "gaussian_bump",
    "two_stream",
    "batched_langmuir",
    "random_tree_flags",
    "random_particles",
    "particle_handling",
    "random_field",
]


def uniform_tree_flags(d: int, depth: int) -> np.ndarray:
    """Level-order flags of the complete tree with every leaf on ``depth``."""
    n_internal = sum(3 ** (l * d) for l in range(depth))
    n_leaves = 3 ** (depth * d)
    return np.concatenate([np.ones(n_internal, np.uint8), np.zeros(n_leaves, np.uint8)])


def _child_offsets(d: int) -> np.ndarray:
    digits = np.arange(3 ** d)
    return np.stack([(digits // 3 ** a) % 3 for a in range(d)], axis=1)  # (3^d, d)


def tree_flags_from_predicate(d: int, max_depth: int, refine) -> np.ndarray:
    """Level-order flags of the tree in which cell (level, coords) is refined
    iff ``level < max_depth and refine(level, coords)``.

    ``refine`` receives the level and an (n, d) int64 array of cell coordinates
    and returns a boolean mask.
    """
    offs = _child_offsets(d)
    coords = np.zeros((1, d), np.int64)
    out = []
    for level in range(max_depth + 1):
        if level == max_depth:
            mask = np.zeros(len(coords), bool)
        else:
            mask = np.asarray(refine(level, coords), bool)
        out.append(mask.astype(np.uint8))
        ref = coords[mask]
        if len(ref) == 0:
            break
        coords = (3 * ref[:, None, :] + offs[None, :, :]).reshape(-1, d)
    return np.concatenate(out)


def random_tree_flags(d: int, max_depth: int, p_refine: float, seed: int,
                      min_depth: int = 0) -> np.ndarray:
    """Random unbalanced tree: every cell above ``min_depth`` is refined, the
    others with probability ``p_refine`` (drawn in level order)."""
    rng = np.random.default_rng(seed)

    def refine(level, coords):
        if level < min_depth:
            return np.ones(len(coords), bool)
        return rng.random(len(coords)) < p_refine

    return tree_flags_from_predicate(d, max_depth, refine)


@dataclass
class Workload:
    """One plasma instance: tree flags, particles and physical parameters."""

    name: str
    d: int
    flags: np.ndarray
    x: np.ndarray            # (d, N) float64 in [0,1)
    v: np.ndarray            # (d, N) float64
    q: float                 # charge per particle
    qm: float                # charge / mass
    ion: float               # ion background density
    dt: float
    steps: int
    k_mode: int = 1          # perturbation wave number (in units of 2*pi)
    vth: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[1])


def _perturbed_coordinate(u: np.ndarray, amp: float, k: int) -> np.ndarray:
    """Invert the CDF of density 1 + amp*cos(2*pi*k*x) on [0,1) (Newton)."""
    x = u.copy()
    w = 2.0 * math.pi * k
    for _ in range(30):
        f = x + amp / w * np.sin(w * x) - u
        x -= f / (1.0 + amp * np.cos(w * x))
    return np.mod(x, 1.0)


def _stratified(n_cells_axis: int, per_axis: int, d: int) -> np.ndarray:
    """Quiet-start lattice: per_axis^d points at the centres of a regular
    sub-lattice of every cell, returned as (d, N) in [0,1)."""
    m = n_cells_axis * per_axis
    g = (np.arange(m, dtype=np.float64) + 0.5) / m
    mesh = np.meshgrid(*([g] * d), indexing="ij")
    return np.stack([mesh[d - 1 - a].reshape(-1) for a in range(d)])  # x fastest


def _normal_quantiles(m: int) -> np.ndarray:
    nd = NormalDist()
    return np.array([nd.inv_cdf((i + 0.5) / m) for i in range(m)])


def langmuir(d: int, depth: int, ppc: int, vth: float = 0.05, amp: float = 0.01,
             k: int = 1, dt: float = 0.1, steps: int = 50, seed: int = 0,
             quiet_v: bool | None = None, name: str = "langmuir") -> Workload:
    """Langmuir-wave start on a uniform tree (configs 2D 27x27 and 3D 243^3).

    Quiet start: ppc must be a perfect d-th power; the sub-lattice x coordinate
    is displaced through the inverse CDF of 1 + amp*cos(2*pi*k*x).  Velocities
    are Maxwellian with standard deviation vth per component (seeded).  With
    ``quiet_v`` (default for N <= 1e7) the x-velocities of every line of equal
    initial x are the Maxwellian quantiles (i + 1/2)/m in a seeded random order,
    so the x-v_x phase space of the k_y = k_z = 0 modes starts noise-free.
    """
    per_axis = round(ppc ** (1.0 / d))
    if per_axis ** d != ppc:
        raise ValueError("ppc must be a perfect d-th power for the quiet start")
    m = 3 ** depth * per_axis
    g = (np.arange(m, dtype=np.float64) + 0.5) / m
    gx = _perturbed_coordinate(g, amp, k)
    # particle index p = ix + m*iy (+ m^2*iz): x fastest
    x = np.empty((d, m ** d))
    x[0] = np.tile(gx, m ** (d - 1))
    if d == 2:
        x[1] = np.repeat(g, m)
    else:
        x[1] = np.tile(np.repeat(g, m), m)
        x[2] = np.repeat(g, m * m)
    n = x.shape[1]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((d, n)) * vth
    if quiet_v is None:
        quiet_v = n <= 10_000_000
    if quiet_v:
        m_line = (3 ** depth * per_axis) ** (d - 1)      # particles sharing one initial x
        n_lines = n // m_line
        vals = _normal_quantiles(m_line) * vth
        order = np.argsort(rng.random((n_lines, m_line)), axis=1)
        # particle index = ix + n_lines * (rest), x fastest
        vx = np.empty(n)
        vx.reshape(m_line, n_lines)[:, :] = vals[order].T
        v[0] = vx
    return Workload(name=name, d=d, flags=uniform_tree_flags(d, depth), x=x, v=v,
                    q=-1.0 / n, qm=-1.0, ion=1.0, dt=dt, steps=steps, k_mode=k, vth=vth,
                    extra={"depth": depth, "ppc": ppc, "amp": amp})


def gaussian_bump(n: int = 1_000_000, d: int = 2, base_depth: int = 4, vth: float = 0.02,
                  sigma: float = 0.1, peak: float = 10.0, tail_frac: float = 0.05,
                  clip_cells: float = 20.0, finest_depth: int = 6, dt: float = 0.1,
                  steps: int = 100, seed: int = 0) -> Workload:
    """Adaptive 2D start: uniform background plus a Gaussian bump (peak = peak x
    background) at the domain centre; Maxwellian velocities plus a Cauchy tail.

    The tree returned is the uniform base tree; the ppc criterion of the method
    refines it.  Tail speeds are clipped to ``clip_cells`` widths of the finest
    admissible cell per step.
    """
    rng = np.random.default_rng(seed)
    bump_mass = (peak - 1.0) * (2.0 * math.pi * sigma * sigma) ** (d / 2.0)
    n_bg = int(round(n / (1.0 + bump_mass)))
    n_bump = n - n_bg
    x_bg = rng.random((d, n_bg))
    x_b = np.mod(0.5 + sigma * rng.standard_normal((d, n_bump)), 1.0)
    x = np.concatenate([x_bg, x_b], axis=1)
    perm = rng.permutation(n)
    x = x[:, perm]
    v = rng.standard_normal((d, n)) * vth
    n_tail = int(round(tail_frac * n))
    idx = rng.choice(n, n_tail, replace=False)
    speed = np.abs(vth * rng.standard_cauchy(n_tail))
    vmax = clip_cells * (3.0 ** -finest_depth) / dt
    speed = np.minimum(speed, vmax)
    dirs = rng.standard_normal((d, n_tail))
    dirs /= np.linalg.norm(dirs, axis=0, keepdims=True)
    v[:, idx] = dirs * speed
    x = np.where(x >= 1.0, 0.0, x)
    return Workload(name="gaussian_bump", d=d, flags=uniform_tree_flags(d, base_depth), x=x,
                    v=v, q=-1.0 / n, qm=-1.0, ion=1.0, dt=dt, steps=steps, vth=vth,
                    extra={"base_depth": base_depth, "ppc_max": 64, "min_depth": base_depth,
                           "max_depth": finest_depth, "retree_every": 10})


def two_stream(n: int = 200_000_000, d: int = 3, base_depth: int = 4, vth_bg: float = 0.05,
               vth_beam: float = 0.01, beam_cells: float = 8.0, beam_frac: float = 0.1,
               dt: float = 0.1, steps: int = 100, seed: int = 0) -> Workload:
    """3D two-stream start: thermal background plus two counter-streaming beams
    along x at +-beam_cells widths of the base-depth-plus-one cell per step."""
    rng = np.random.default_rng(seed)
    x = rng.random((d, n))
    v = rng.standard_normal((d, n)) * vth_bg
    nb = int(round(beam_frac * n))
    ub = beam_cells * (3.0 ** -(base_depth + 1)) / dt
    v[:, :nb] = rng.standard_normal((d, nb)) * vth_beam
    v[0, :nb] += ub
    v[:, nb:2 * nb] = rng.standard_normal((d, nb)) * vth_beam
    v[0, nb:2 * nb] -= ub
    return Workload(name="two_stream", d=d, flags=uniform_tree_flags(d, base_depth), x=x, v=v,
                    q=-1.0 / n, qm=-1.0, ion=1.0, dt=dt, steps=steps, vth=vth_bg,
                    extra={"base_depth": base_depth, "ppc_max": 32, "min_depth": base_depth,
                           "max_depth": base_depth + 2, "retree_every": 5})


def batched_langmuir(n_inst: int = 256, n_min: int = 1000, n_max: int = 1_000_000,
                     dt: float = 0.1, steps: int = 100, amp: float = 0.01,
                     scale: float = 1.0) -> list[Workload]:
    """Uneven batch of 2D Langmuir instances; instance i draws from seed i.

    Particle counts are log-uniform in [n_min, n_max] (times ``scale``), depths
    uniform in {3,4,5}, vth uniform in [0.02, 0.1], mode k in {1,2,4}.
    """
    out = []
    for i in range(n_inst):
        rng = np.random.default_rng(i)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale))
        n = max(n, 16)
        depth = int(rng.integers(3, 6))
        vth = float(rng.uniform(0.02, 0.1))
        k = int(rng.choice([1, 2, 4]))
        u = (np.arange(n, dtype=np.float64) + rng.random(n)) / n
        x0 = _perturbed_coordinate(u, amp, k)
        x1 = rng.random(n)
        x = np.stack([x0, x1])
        v = rng.standard_normal((2, n)) * vth
        out.append(Workload(name=f"inst{i}", d=2, flags=uniform_tree_flags(2, depth), x=x, v=v,
                            q=-1.0 / n, qm=-1.0, ion=1.0, dt=dt, steps=steps, k_mode=k,
                            vth=vth, extra={"depth": depth}))
    return out


def particle_handling(d: int, n: int, dam: bool = False, seed: int = 0, base_depth: int = 1) -> Workload:
    """The particle-handling workload of the paper's experiments (Section 6):
    no field; positions uniform in the unit box, or in the corner (0, 0.1)^d
    ("breaking dam", dam=True); velocities of uniformly distributed speed
    0 <= |v| <= 1 in a uniformly random direction.  The tree returned is the
    uniform base tree; the ppc criterion refines it."""
    rng = np.random.default_rng(seed)
    x = rng.random((d, n)) * (0.1 if dam else 1.0)
    dirs = rng.standard_normal((d, n))
    dirs /= np.linalg.norm(dirs, axis=0, keepdims=True)
    v = dirs * rng.random(n)[None, :]
    return Workload(name="particle_handling_dam" if dam else "particle_handling", d=d,
                    flags=uniform_tree_flags(d, base_depth), x=x, v=v, q=0.0, qm=0.0, ion=0.0, dt=1e-3,
                    steps=10, extra={"dam": dam, "base_depth": base_depth})


def thermal_plasma(d: int = 2, depth: int = 5, ppc: int = 100, dt: float = 0.01, seed: int = 0) -> Workload:
    """The validation plasma of Appendix A: a uniform grid of 3^depth cells per
    axis whose cell is one Debye length, ppc particles per cell at uniformly
    random positions, Maxwellian velocities of thermal speed v_th = lambda_D
    omega_p per component (one cell width per plasma time), q/m = -1 and a
    neutralising ion background; omega_p dt = 0.01.  The random start seeds a
    sea of Langmuir waves at every wave vector."""
    rng = np.random.default_rng(seed)
    n = ppc * 3 ** (depth * d)
    x = rng.random((d, n))
    v = rng.standard_normal((d, n)) * (1.0 / 3 ** depth)
    return Workload(name="thermal_plasma", d=d, flags=uniform_tree_flags(d, depth), x=x, v=v, q=-1.0 / n,
                    qm=-1.0, ion=1.0, dt=dt, steps=0, extra={"vth": 1.0 / 3 ** depth, "ppc": ppc})


def random_particles(d: int, n: int, seed: int, vmax: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Uniform positions in [0,1)^d and velocities uniform in [-vmax, vmax]^d."""
    rng = np.random.default_rng(seed)
    x = rng.random((d, n))
    v = rng.uniform(-vmax, vmax, (d, n))
    return x, v


def random_field(d: int, n_vertices: int, seed: int, amp: float) -> np.ndarray:
    """A seeded vertex field for tests that hold E fixed: FP32 values uniform
    in [-amp, amp), shape (d, n_vertices) in the vertex numbering of the tree."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, (d, n_vertices)).astype(np.float32)
