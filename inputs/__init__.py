"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module produces the *data* the method is run on -- U(1) gauge fields,
the random start vectors of the multigrid setup, and the named workloads --
and nothing of the method's own arithmetic.  The Z2 noise drawn by the
Hutchinson estimator is *not* produced here: the oracle and the CUDA path each
implement that counter-based generator independently.

Randomness comes from a counter-based stream built on the splitmix64 output
function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), so every value is a pure function of
(seed, stream, index) and identical on every machine and numpy version.

The paper (Sect. 4.3) runs on "the exact same Schwinger matrix" of its
predecessor, which is not available; Metropolis U(1) fields of the same
lattice sizes stand in for it.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

__all__ = [
    "uniform", "gaussian_complex", "metropolis_u1", "start_vectors",
    "Workload", "WORKLOADS", "workload",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_S30, _S27, _S31, _S11 = (np.uint64(s) for s in (30, 27, 31, 11))


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GAMMA)
        return _mix((k ^ np.uint64(stream & 0xFFFFFFFFFFFFFFFF)) + _GAMMA)


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the splitmix64 sequence started at key(seed, stream)."""
    key = _key(seed, stream)
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(key + i * _GAMMA)
    return (z >> _S11).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_complex(seed: int, stream: int, shape) -> np.ndarray:
    """Complex normal entries with E|z|^2 = 1 (Box-Muller on two uniform streams)."""
    n = int(np.prod(shape))
    u1 = uniform(seed, 2 * stream, n)
    u2 = uniform(seed, 2 * stream + 1, n)
    r = np.sqrt(-np.log1p(-u1))          # |z| for E|z|^2 = 1
    z = r * np.exp(2j * math.pi * u2)
    return z.reshape(shape)


def _uniform_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Entries idx of uniform(seed, stream, .): the same counter-based values."""
    key = _key(seed, stream)
    i = idx.astype(np.uint64) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = _mix(key + i * _GAMMA)
    return (z >> _S11).astype(np.float64) * (1.0 / 9007199254740992.0)


def _metropolis_rows(th, t_i, x_i, mu, beta, delta, seed, stream):
    """One Metropolis hit on the links (t_i, x_i, mu) of th (in place); every value
    is computed exactly as in the whole-lattice form of metropolis_u1."""
    Lt, Lx, _ = th.shape
    t0, t1 = th[..., 0], th[..., 1]
    tp, tm = (t_i + 1) % Lt, (t_i - 1) % Lt
    xp, xm = (x_i + 1) % Lx, (x_i - 1) % Lx
    if mu == 0:
        a = t1[t_i, xp] - t0[tp, x_i] - t1[t_i, x_i]
        b = t0[tm, x_i] + t1[tm, xp] - t1[tm, x_i]
        cur = t0[t_i, x_i]
    else:
        a = t0[t_i, x_i] + t1[t_i, xp] - t0[tp, x_i]
        b = t0[t_i, xm] - t0[tp, xm] - t1[t_i, xm]
        cur = t1[t_i, x_i]
    flat = t_i * Lx + x_i
    u_prop = _uniform_at(seed, stream, flat)
    u_acc = _uniform_at(seed, stream + 1, flat)
    new = cur + delta * (2.0 * u_prop - 1.0)
    if mu == 0:
        s_old = -np.cos(cur + a) - np.cos(b - cur)
        s_new = -np.cos(new + a) - np.cos(b - new)
    else:
        s_old = -np.cos(a - cur) - np.cos(b + cur)
        s_new = -np.cos(a - new) - np.cos(b + new)
    dS = beta * (s_new - s_old)
    accept = u_acc < np.exp(-np.maximum(dS, 0.0))
    th[t_i, x_i, mu] = np.where(accept, np.remainder(new + math.pi, 2 * math.pi) - math.pi, cur)


def _metropolis_worker(shm_name, shape, r0, r1, beta, sweeps, seed, delta, barrier):
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=shm_name)
    try:
        th = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
        Lt, Lx, _ = shape
        tt, xx = np.meshgrid(np.arange(r0, r1), np.arange(Lx), indexing="ij")
        sel = {}
        for mu in (0, 1):
            for parity in (0, 1):
                t_i, x_i = np.nonzero(((tt if mu == 0 else xx) % 2) == parity)
                sel[(mu, parity)] = (t_i + r0, x_i)
        stream = 1
        for _ in range(sweeps):
            for mu in (0, 1):
                for parity in (0, 1):
                    _metropolis_rows(th, *sel[(mu, parity)], mu, beta, delta, seed, stream)
                    stream += 2
                    barrier.wait()
        del th
    finally:
        shm.close()


def _metropolis_parallel(Lx, Lt, beta, sweeps, seed, delta, workers):
    """metropolis_u1 with the time rows split over `workers` processes.  Within one
    (mu, parity) sub-step no updated link enters another updated link's action, so
    the strips update a shared array independently between barriers; the result is
    the serial one bit for bit."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    ctx = mp.get_context("spawn")      # safe after CUDA initialisation in the parent
    shape = (Lt, Lx, 2)
    shm = shared_memory.SharedMemory(create=True, size=int(np.prod(shape)) * 8)
    try:
        th = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
        th[:] = (2.0 * uniform(seed, 0, Lt * Lx * 2) - 1.0).reshape(shape) * math.pi
        barrier = ctx.Barrier(workers, timeout=3600)
        bounds = np.linspace(0, Lt, workers + 1).astype(int)
        procs = [ctx.Process(target=_metropolis_worker,
                             args=(shm.name, shape, int(bounds[w]), int(bounds[w + 1]), beta, sweeps, seed, delta,
                                   barrier)) for w in range(workers)]
        for p in procs:
            p.start()
        for p in procs:
            p.join()
        if any(p.exitcode != 0 for p in procs):
            raise RuntimeError("metropolis_u1: a worker process failed")
        out = th.copy()
        del th
        return out
    finally:
        shm.close()
        shm.unlink()


def metropolis_u1(Lx: int, Lt: int, beta: float, sweeps: int, seed: int,
                  delta: float = 1.0, workers: int | None = None) -> np.ndarray:
    """U(1) link angles theta[t, x, mu] from a seeded Metropolis run.

    Action S = beta * sum_x (1 - cos theta_P(x)) with the plaquette angle
    theta_P(x) = th0(x) + th1(x+e0) - th0(x+e1) - th1(x); mu = 0 is space (x),
    mu = 1 is time (t); the gauge field is periodic in both directions.
    Hot start, one Metropolis hit per link and sweep with proposal
    theta' = theta + delta * (2u - 1).  Links that share no plaquette are
    updated together (x-links by parity of t, t-links by parity of x).
    Lattices of 2^18 sites or more are generated by several host processes
    (`workers`, default: the host's cores, at most 16) with the same result.
    """
    if workers is None:
        workers = 1 if Lx * Lt < (1 << 18) else max(1, min(16, os.cpu_count() or 1))
    workers = min(workers, Lt // 2)
    if workers > 1 and Lt % 2 == 0:
        return _metropolis_parallel(Lx, Lt, beta, sweeps, seed, delta, workers)
    th = (2.0 * uniform(seed, 0, Lt * Lx * 2) - 1.0).reshape(Lt, Lx, 2) * math.pi
    tpar = (np.arange(Lt) % 2)[:, None] * np.ones((1, Lx), dtype=np.int64)
    xpar = np.ones((Lt, 1), dtype=np.int64) * (np.arange(Lx) % 2)[None, :]
    stream = 1
    for _ in range(sweeps):
        for mu in (0, 1):
            for parity in (0, 1):
                mask = (tpar if mu == 0 else xpar) == parity
                t0, t1 = th[..., 0], th[..., 1]
                if mu == 0:
                    # th0(x,t) enters P(x,t) with + and P(x,t-1) with -.
                    a = np.roll(t1, -1, axis=1) - np.roll(t0, -1, axis=0) - t1
                    b = (np.roll(t0, 1, axis=0) + np.roll(np.roll(t1, -1, axis=1), 1, axis=0)
                         - np.roll(t1, 1, axis=0))
                    cur = t0
                else:
                    # th1(x,t) enters P(x,t) with - and P(x-1,t) with +.
                    a = t0 + np.roll(t1, -1, axis=1) - np.roll(t0, -1, axis=0)
                    b = (np.roll(t0, 1, axis=1) - np.roll(np.roll(t0, -1, axis=0), 1, axis=1)
                         - np.roll(t1, 1, axis=1))
                    cur = t1
                u_prop = uniform(seed, stream, Lt * Lx).reshape(Lt, Lx)
                u_acc = uniform(seed, stream + 1, Lt * Lx).reshape(Lt, Lx)
                stream += 2
                new = cur + delta * (2.0 * u_prop - 1.0)
                if mu == 0:
                    s_old = -np.cos(cur + a) - np.cos(b - cur)
                    s_new = -np.cos(new + a) - np.cos(b - new)
                else:
                    s_old = -np.cos(a - cur) - np.cos(b + cur)
                    s_new = -np.cos(a - new) - np.cos(b + new)
                dS = beta * (s_new - s_old)
                accept = mask & (u_acc < np.exp(-np.maximum(dS, 0.0)))
                new = np.where(accept, np.remainder(new + math.pi, 2 * math.pi) - math.pi, cur)
                th[..., mu] = new
    return th


def start_vectors(seed: int, level: int, n: int, nvec: int) -> np.ndarray:
    """Complex Gaussian start vectors of the multigrid setup, shape (nvec, n)."""
    return gaussian_complex(seed, 1000 + level, (nvec, n))


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload (lattice, gauge recipe, hierarchy, sampling)."""
    name: str
    Lx: int
    Lt: int
    beta: float
    m0: float
    agg: tuple            # ((ax, at), ...) per coarsening step
    nvec: tuple           # test vectors per spin, per coarsening step
    k: int                # deflated triplets of the coarsest operator
    nrhs: int             # Z2 samples per level in one block
    setup_iters: int = 4
    sweeps: int = 200
    gauge_seed: int = 1
    noise_seed: int = 2
    setup_seed: int = 3
    skip: tuple = ()      # levels left out of the telescoping sum (the last ones: solver-only levels)
    kcycle: int = 0       # K-cycle steps per coarse-grid correction (0: V-cycle)
    defl_tol: float = 1e-9
    defl_iters: int = 400

    @property
    def nlevels(self) -> int:
        return len(self.agg) + 1

    @property
    def term_levels(self) -> tuple:
        """Levels (1-based) that start a term of the telescoping sum."""
        return tuple(lev for lev in range(1, self.nlevels + 1) if lev not in self.skip)

    @property
    def nterms(self) -> int:
        return len(self.term_levels)

    @property
    def n1(self) -> int:
        return 2 * self.Lx * self.Lt

    def gauge(self) -> np.ndarray:
        return metropolis_u1(self.Lx, self.Lt, self.beta, self.sweeps, self.gauge_seed)

    def level_dims(self):
        """[(Lx_l, Lt_l, dof_per_site_l)] for l = 1..L."""
        dims = [(self.Lx, self.Lt, 2)]
        for (ax, at), nv in zip(self.agg, self.nvec):
            lx, lt, _ = dims[-1]
            dims.append((lx // ax, lt // at, 2 * nv))
        return dims

    def start_vectors(self):
        """Per coarsening step l: (nvec_l, n_l) complex start vectors."""
        out = []
        for lev, ((lx, lt, d), nv) in enumerate(zip(self.level_dims()[:-1], self.nvec), start=1):
            out.append(start_vectors(self.setup_seed, lev, lx * lt * d, nv))
        return out


# Near-critical mass of the 1024^2 workload: sigma_min(D) ~ 1e-3 on the 256^2 field of
# the same recipe (python -m oracle.tune_mass schwinger-1024x1024 1e-3 --lattice 256).
M0_1024 = -0.081836

# Mass of the 128^2 workload: chosen with the oracle so that sigma_min(D) ~ 1e-3
# (value written by oracle/tune_mass.py into tests/golden/mass_128.json).
WORKLOADS = {
    "tiny-8x8": Workload("tiny-8x8", 8, 8, 3.0, -0.10, ((2, 2),), (2,), 4, 8,
                         sweeps=20),
    "schwinger-16x16": Workload("schwinger-16x16", 16, 16, 3.0, -0.10, ((4, 4),), (4,), 16, 64,
                                gauge_seed=1001, noise_seed=2001, setup_seed=3001),
    "schwinger-128x128": Workload("schwinger-128x128", 128, 128, 3.0, -0.141406,
                                  ((4, 4), (2, 2)), (8, 8), 64, 256,
                                  gauge_seed=2001, noise_seed=4001, setup_seed=6001),
    # 3-term sum (levels 1..3, 65536 / 16384 coarse unknowns on levels 2 / 3) with one
    # solver-only level below (16^2 sites x 16 = 4096 unknowns, stored inverse)
    "schwinger-256x256": Workload("schwinger-256x256", 256, 256, 5.0, -0.05,
                                  ((4, 4), (2, 2), (2, 2)), (8, 8, 8), 128, 512,
                                  gauge_seed=3001, noise_seed=6001, setup_seed=9001, skip=(4,)),
    # 3-term sum (n = 2097152 / 1048576 / 262144 on levels 1..3) with one solver-only
    # level (4x4 aggregates of level 3: 32^2 sites x 16 = 16384 unknowns, stored
    # inverse), so that the level-3 solves are two-grid solves with an exact coarse
    # correction; m0 tuned with the oracle on a 256^2 field of the same recipe
    # (tests/golden/mass_1024_at256.json)
    "schwinger-1024x1024": Workload("schwinger-1024x1024", 1024, 1024, 5.0, M0_1024,
                                    ((4, 4), (2, 2), (4, 4)), (8, 8, 8), 512, 128,
                                    gauge_seed=4001, noise_seed=8001, setup_seed=12001, skip=(4,),
                                    defl_tol=1e-3, defl_iters=16),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
