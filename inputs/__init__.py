"""Seeded synthetic inputs for the particle-SMC workloads.

This module only *generates data*: observation sequences, phylogenies and
run/request mixes.  It holds none of the SMC method's arithmetic (no
weighting, no resampling, no model blocks) and is imported by the tests, the
benchmark and the oracle harness alike, so that the CUDA path and the CPU
oracle are fed byte-identical inputs.

Stand-ins (the paper's datasets are not available):
  * the Alcedinidae / Tyrant-flycatcher phylogenies of the CRBD experiments
    (Section 6.1 / 6.3) -> seeded Yule trees rescaled to height 1.0;
  * observation sequences -> simulated from the linear-Gaussian state-space
    model itself (the Eq. 2 family).

All generators use numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

__all__ = [
    "Tree",
    "yule_tree",
    "two_tip_tree",
    "lg_observations",
    "RunSpec",
    "batch_specs",
    "poisson_arrivals",
    "random_logw",
]


@dataclass
class Tree:
    """A rooted binary tree in array form (root is node 0).

    parent[v] = -1 for the root; left[v] = right[v] = -1 for tips.
    age[v] is the time before the present (tips at 0, root at `root_age`).
    preorder lists every node, root first, left subtree before right.
    """

    parent: np.ndarray  # int32 [M]
    left: np.ndarray  # int32 [M]
    right: np.ndarray  # int32 [M]
    age: np.ndarray  # float64 [M]
    preorder: np.ndarray  # int32 [M]

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    @property
    def n_tips(self) -> int:
        return (self.n_nodes + 1) // 2

    def max_depth(self) -> int:
        """Number of edges on the longest root-to-tip path."""
        depth = np.zeros(self.n_nodes, dtype=np.int64)
        for v in self.preorder[1:]:
            depth[v] = depth[self.parent[v]] + 1
        return int(depth.max())

    def max_pending_right(self) -> int:
        """Largest number of right children that are pending at once during a
        left-first preorder walk (the depth a pending-rate stack needs)."""
        best = 0
        pend = 0
        for v in self.preorder:
            p = self.parent[v]
            if p >= 0 and self.right[p] == v:
                pend -= 1
            if self.left[v] >= 0:
                pend += 1
            best = max(best, pend)
        return best


def _preorder(left: np.ndarray, right: np.ndarray) -> np.ndarray:
    out = []
    stack = [0]
    while stack:
        v = stack.pop()
        out.append(v)
        if right[v] >= 0:
            stack.append(int(right[v]))
        if left[v] >= 0:
            stack.append(int(left[v]))
    return np.asarray(out, dtype=np.int32)


def yule_tree(n_tips: int, seed: int, height: float = 1.0) -> Tree:
    """Seeded pure-birth (Yule, rate 1) tree with `n_tips` tips.

    Starts from two lineages at the root; with k lineages alive the waiting
    time is Exp(k) and a uniformly chosen lineage splits.  When n lineages are
    reached one more Exp(n) interval is added so that no tip branch has zero
    length.  Ages are then rescaled so the root age equals `height`.
    """
    if n_tips < 2:
        raise ValueError("a tree needs at least two tips")
    rng = np.random.Generator(np.random.PCG64(seed))
    m = 2 * n_tips - 1
    parent = np.full(m, -1, dtype=np.int32)
    left = np.full(m, -1, dtype=np.int32)
    right = np.full(m, -1, dtype=np.int32)
    birth = np.zeros(m, dtype=np.float64)  # forward time at which node's lower end occurs
    next_id = 1
    # lineage = the child node id whose branch is still growing
    lineages = []
    for _ in range(2):
        c = next_id
        next_id += 1
        parent[c] = 0
        lineages.append(c)
    left[0], right[0] = lineages[0], lineages[1]
    t = 0.0
    while len(lineages) < n_tips:
        k = len(lineages)
        t += rng.exponential(1.0 / k)
        j = int(rng.integers(k))
        v = lineages[j]
        birth[v] = t  # v becomes an internal node at time t
        a, b = next_id, next_id + 1
        next_id += 2
        parent[a] = v
        parent[b] = v
        left[v], right[v] = a, b
        lineages[j] = a
        lineages.append(b)
    t += rng.exponential(1.0 / n_tips)
    for v in lineages:
        birth[v] = t
    age = (t - birth) * (height / t)
    age[0] = height
    for v in lineages:
        age[v] = 0.0
    return Tree(parent, left, right, age, _preorder(left, right))


def two_tip_tree(root_age: float = 1.0) -> Tree:
    parent = np.array([-1, 0, 0], dtype=np.int32)
    left = np.array([1, -1, -1], dtype=np.int32)
    right = np.array([2, -1, -1], dtype=np.int32)
    age = np.array([root_age, 0.0, 0.0])
    return Tree(parent, left, right, age, np.array([0, 1, 2], dtype=np.int32))


def lg_observations(T: int, seed: int, a: float = 0.9, b: float = 0.0,
                    q_sd: float = 1.0, r_sd: float = 0.5,
                    x0_mean: float = 0.0, x0_sd: float = 1.0) -> np.ndarray:
    """Simulate y_1..y_T from x0~N(x0_mean,x0_sd^2), x_t=a x_{t-1}+b+N(0,q_sd^2),
    y_t=x_t+N(0,r_sd^2).  Returns float64 [T]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = x0_mean + x0_sd * rng.standard_normal()
    y = np.empty(T, dtype=np.float64)
    for t in range(T):
        x = a * x + b + q_sd * rng.standard_normal()
        y[t] = x + r_sd * rng.standard_normal()
    return y


@dataclass
class RunSpec:
    """One independent SMC run of a mixed batch or request stream."""

    kind: str  # "lg" or "crbd"
    n_particles: int
    seed: int
    T: int = 0  # lg: number of observations
    obs_seed: int = 0
    tips: int = 0  # crbd: tips of its own Yule tree
    tree_seed: int = 0

    def n_segments(self) -> int:
        return self.T if self.kind == "lg" else 2 * self.tips - 1

    def particle_steps(self) -> int:
        return self.n_particles * self.n_segments()


def _log_uniform_int(rng, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def batch_specs(n_runs: int = 512, seed: int = 4, n_lo: int = 256,
                n_hi: int = 65536) -> list[RunSpec]:
    """Mixed batch: half linear-Gaussian runs (T log-uniform in 20..500), half
    CRBD runs (tips log-uniform in 16..256); N log-uniform in n_lo..n_hi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n_runs):
        n = _log_uniform_int(rng, n_lo, n_hi)
        if i % 2 == 0:
            T = _log_uniform_int(rng, 20, 500)
            specs.append(RunSpec("lg", n, seed=1000 + i, T=T, obs_seed=5000 + i))
        else:
            tips = _log_uniform_int(rng, 16, 256)
            specs.append(RunSpec("crbd", n, seed=1000 + i, tips=tips, tree_seed=9000 + i))
    return specs


def poisson_arrivals(rate: float, duration: float, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream with the given mean rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        out.append(t)
    return np.asarray(out)


def random_logw(n: int, seed: int, scale: float = 3.0, dead_frac: float = 0.0) -> np.ndarray:
    """Log-weights for resampling-primitive tests: normal with the given scale,
    with an optional fraction of particles at -inf (killed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lw = scale * rng.standard_normal(n)
    if dead_frac > 0:
        lw[rng.random(n) < dead_frac] = -np.inf
    return lw


def seir_observations(n_days: int = 182, seed: int = 7, report_every: int = 7) -> np.ndarray:
    """Daily report series for the vector-borne disease SEIR model (stand-in for
    the dengue case data, which is not available): the model run forward with
    fixed parameters (human attack 0.3, incubation 1/4.4, recovery 1/4.5,
    mosquito attack 0.3, mosquito incubation 1/6.5, reporting 0.6; 6 infectious,
    5 exposed, 7,370 humans, 3 mosquitoes per human) by numpy's generator.  New
    infectious cases accumulate and a report y ~ Binomial(cases, 0.6) is made
    every `report_every` days (days report_every - 1, 2 report_every - 1, ...);
    other days hold -1 (no report).  Float array of length n_days."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h_lam, h_del, h_gam, m_lam, m_del, rho = 0.3, 1 / 4.4, 1 / 4.5, 0.3, 1 / 6.5, 0.6
    n = 7370
    hS, hE, hI, hR = n - 11, 5, 6, 0
    mS, mE, mI, mR = 3 * n, 0, 0, 0
    y = np.full(n_days, -1.0)
    z = hI
    for t in range(n_days):
        if t > 0:
            hN = hS + hE + hI + hR
            tau = rng.binomial(hS, 1.0 - np.exp(-mI / hN))
            dE = rng.binomial(tau, h_lam)
            dI = rng.binomial(hE, h_del)
            dR = rng.binomial(hI, h_gam)
            m_tau = rng.binomial(mS, 1.0 - np.exp(-hI / hN))
            mN = mS + mE + mI + mR
            mdE = rng.binomial(m_tau, m_lam)
            mdI = rng.binomial(mE, m_del)
            hS, hE, hI, hR = hS - dE, hE + dE - dI, hI + dI - dR, hR + dR
            mS, mE, mI = mS - mdE, mE + mdE - mdI, mI + mdI
            mS, mE, mI, mR = (rng.binomial(mS, 6 / 7), rng.binomial(mE, 6 / 7),
                              rng.binomial(mI, 6 / 7), rng.binomial(mR, 6 / 7))
            mS += rng.binomial(mN, 1 / 7)
            z += dI
        if (t + 1) % report_every == 0:
            y[t] = float(rng.binomial(z, rho))
            z = 0
    return y
