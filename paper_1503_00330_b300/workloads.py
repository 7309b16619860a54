"""Seeded synthetic workloads for the PI^2-RH / LWPR hot path.

This module only draws inputs: it holds none of the method's arithmetic, and
both the CUDA path and the FP64 oracle consume exactly the arrays it returns.
Everything is drawn in float64 with ``numpy.random.Generator(PCG64(seed))`` in
the fixed order documented per function, then rounded ONCE to float32; the
oracle widens those float32 values exactly.

The paper's trained quadrotor LWPR models (3 outputs over 4 inputs with 15, 15
and 24 receptive fields, Sec. 4.1) and its flight data are not available, so
these quadrotor-shaped stand-ins are used instead: a 12-dim state (position,
velocity, roll/pitch/yaw, body rates), a 4-dim control (thrust, roll, pitch,
yaw-rate), and an LWPR model with 12 outputs (state derivatives) over the
16-dim input z = [x, u].

Named workloads (sizes in rollouts K, steps T, fields per output L):
  * ``small``     K=256,   T=50,  L=64,   4 obstacles  (oracle-sized)
  * ``realtime``  K=8192,  T=100, L=512,  16 obstacles, 20 receding-horizon
                  iterations with warm-start shift, seed per iteration = seed + it
  * ``precision`` K=65536, T=100, L=2048, D_j with condition numbers log-uniform
                  in [1, 1e3]
  * ``batched``   64 controllers, K ~ logU[1024, 32768], T ~ U{30..150},
                  L ~ logU[128, 2048], own parameters, obstacles and seed each
  * ``serving``   256 quadrotors, Poisson arrivals at 50 Hz each,
                  K ~ U{2048..16384}, T ~ U{50..120}, one shared L=1024 model
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

NX, NU, NZ, NY = 12, 4, 16, 12


@dataclass
class LwprModel:
    """LWPR parameters, float32, row-major.

    c [NY, L, NZ] centers; D [NY, L, NZ, NZ] symmetric distance metrics;
    beta [NY, L, NZ] local slopes; b [NY, L] local offsets (value at the
    center); sigma [NY, L] per-field noise standard deviations; dt Euler step.
    """
    c: np.ndarray
    D: np.ndarray
    beta: np.ndarray
    b: np.ndarray
    sigma: np.ndarray
    dt: np.float32

    @property
    def L(self) -> int:
        return int(self.c.shape[1])


@dataclass
class CostParams:
    """Obstacle-navigation cost (float32 scalars).

    obs_kind 0: w_obs * 1[inside any cylinder]; obs_kind 1 (the paper's Sec. 5
    form): w_obs * sum_i exp(-obs_sharp * d_i^2), with w_crash * 1[inside].
    """
    goal: tuple = (1.5, 1.5, 1.0)
    Q_pos: tuple = (1.0, 1.0, 1.0)
    Q_vel: float = 0.0
    Q_ang: float = 0.0
    w_obs: float = 1.0e3
    obs_sharp: float = 10.0
    radius: float = 0.3
    w_crash: float = 0.0
    w_var: float = 1.0
    w_T: float = 1.0
    obs_kind: int = 0
    obs_xy: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.float32))

    def rounded(self) -> "CostParams":
        f = lambda v: float(np.float32(v))
        return replace(self, goal=tuple(map(f, self.goal)), Q_pos=tuple(map(f, self.Q_pos)),
                       Q_vel=f(self.Q_vel), Q_ang=f(self.Q_ang), w_obs=f(self.w_obs),
                       obs_sharp=f(self.obs_sharp), radius=f(self.radius), w_crash=f(self.w_crash),
                       w_var=f(self.w_var), w_T=f(self.w_T),
                       obs_xy=np.asarray(self.obs_xy, np.float32).reshape(-1, 2))


@dataclass
class Problem:
    """One control update's inputs."""
    model: LwprModel
    cost: CostParams
    x0: np.ndarray        # [NX] float32
    u_nom: np.ndarray     # [T, NU] float32
    K: int
    T: int
    lam: float            # float32-representable
    sigma_u: np.ndarray   # [NU] float32 variances
    seed: int
    M: int = 1
    model_noise: bool = True


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_lwpr(L: int, seed: int, conditioned: bool = False, dt: float = 0.02) -> LwprModel:
    """Draw an LWPR model with L fields per output.

    Draw order: c ~ N(0, I); then D; then beta ~ N(0, 0.3^2); b ~ N(0, 0.1^2);
    sigma ~ U(0.01, 0.1).  D (default): diag(U(0.5, 5)) + 0.1 V V^T with
    V in R^{16x2} ~ N(0, 1).  D (``conditioned``): Q diag(s) Q^T with Q Haar
    orthogonal (QR of a Gaussian with the sign of R's diagonal folded in),
    s_max ~ U(0.5, 5), kappa ~ logU[1, 1e3], and eigenvalues log-uniform in
    [s_max/kappa, s_max] with both ends forced in, so cond(D) = kappa.
    """
    g = _rng(seed)
    n = NY * L
    c = g.standard_normal((n, NZ))
    if not conditioned:
        diag = g.uniform(0.5, 5.0, (n, NZ))
        V = g.standard_normal((n, NZ, 2))
        D = np.einsum("fi,ij->fij", diag, np.eye(NZ)) + 0.1 * np.einsum("fia,fja->fij", V, V)
    else:
        G = g.standard_normal((n, NZ, NZ))
        Qm, R = np.linalg.qr(G)
        Qm = Qm * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
        s_max = g.uniform(0.5, 5.0, n)
        kappa = np.exp(g.uniform(0.0, np.log(1e3), n))
        logs = g.uniform(0.0, 1.0, (n, NZ))
        logs[:, 0], logs[:, 1] = 0.0, 1.0
        s = s_max[:, None] * np.exp(-np.log(kappa)[:, None] * logs)
        D = np.einsum("fik,fk,fjk->fij", Qm, s, Qm)
        D = 0.5 * (D + np.transpose(D, (0, 2, 1)))
    beta = 0.3 * g.standard_normal((n, NZ))
    b = 0.1 * g.standard_normal(n)
    sigma = g.uniform(0.01, 0.1, n)
    f32 = lambda a, shape: np.ascontiguousarray(a.reshape(shape).astype(np.float32))
    return LwprModel(c=f32(c, (NY, L, NZ)), D=f32(D, (NY, L, NZ, NZ)), beta=f32(beta, (NY, L, NZ)),
                     b=f32(b, (NY, L)), sigma=f32(sigma, (NY, L)), dt=np.float32(dt))


def make_obstacles(n_obs: int, seed: int) -> np.ndarray:
    """Cylinder centers ~ U([-2, 2]^2), drawn from their own stream (seed, 1)."""
    g = np.random.Generator(np.random.PCG64([seed, 1]))
    return g.uniform(-2.0, 2.0, (n_obs, 2)).astype(np.float32)


def make_cost(n_obs: int, seed: int, **kw) -> CostParams:
    return CostParams(obs_xy=make_obstacles(n_obs, seed), **kw).rounded()


def paper_cost(n_obs: int = 3, seed: int = 0) -> CostParams:
    """The Sec. 5 experiment cost: (x-W)^2 + (y-W)^2 + 10 (z-W)^2 + angles/5 +
    velocities/10 + 100 sum exp(-10 d^2) + 10 C, with zero terminal cost and no
    variance term."""
    return CostParams(Q_pos=(1.0, 1.0, 10.0), Q_vel=0.1, Q_ang=0.2, w_obs=100.0, obs_sharp=10.0,
                      w_crash=10.0, w_var=0.0, w_T=0.0, obs_kind=1,
                      obs_xy=make_obstacles(n_obs, seed)).rounded()


SIGMA_U = np.array([0.1, 0.05, 0.05, 0.05], np.float32)


def problem(K: int, T: int, L: int, seed: int = 0, n_obs: int = 4, conditioned: bool = False,
            M: int = 1, model_noise: bool = True, cost: CostParams | None = None,
            lam: float = 1.0, model: LwprModel | None = None) -> Problem:
    """A single-controller update with x0 = 0 and u_nom = 0."""
    return Problem(model=model if model is not None else make_lwpr(L, seed, conditioned),
                   cost=cost if cost is not None else make_cost(n_obs, seed),
                   x0=np.zeros(NX, np.float32), u_nom=np.zeros((T, NU), np.float32), K=K, T=T,
                   lam=float(np.float32(lam)), sigma_u=SIGMA_U.copy(), seed=seed, M=M,
                   model_noise=model_noise)


def small(seed: int = 0) -> Problem:
    return problem(256, 50, 64, seed, n_obs=4)


def realtime(seed: int = 0) -> Problem:
    return problem(8192, 100, 512, seed, n_obs=16)


REALTIME_ITERS = 20


def precision(seed: int = 0, K: int = 65536) -> Problem:
    return problem(K, 100, 2048, seed, n_obs=16, conditioned=True)


def batched_sizes(n: int = 64, seed: int = 0):
    """(K, T, L) per controller: K ~ logU[1024, 32768], T ~ U{30..150},
    L ~ logU[128, 2048] (rounded to integers)."""
    g = np.random.Generator(np.random.PCG64([seed, 3]))
    K = np.rint(np.exp(g.uniform(np.log(1024), np.log(32768), n))).astype(int)
    T = g.integers(30, 151, n)
    L = np.rint(np.exp(g.uniform(np.log(128), np.log(2048), n))).astype(int)
    return [(int(k), int(t), int(l)) for k, t, l in zip(K, T, L)]


def batched(n: int = 64, seed: int = 0, scale_K: float = 1.0) -> list[Problem]:
    """Independent controllers, controller i drawn with seed i (own parameters,
    obstacles and noise)."""
    out = []
    for i, (K, T, L) in enumerate(batched_sizes(n, seed)):
        out.append(problem(max(1, int(K * scale_K)), T, L, seed=i, n_obs=16))
    return out


def serving_requests(n_quad: int = 256, rate_hz: float = 50.0, duration_s: float = 1.0,
                     seed: int = 0):
    """Poisson request stream: list of (arrival_s, quad_id, K, T), sorted."""
    g = np.random.Generator(np.random.PCG64([seed, 4]))
    reqs = []
    for q in range(n_quad):
        t = g.exponential(1.0 / rate_hz)
        while t < duration_s:
            reqs.append((float(t), q, int(g.integers(2048, 16385)), int(g.integers(50, 121))))
            t += g.exponential(1.0 / rate_hz)
    reqs.sort()
    return reqs
