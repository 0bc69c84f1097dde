"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no finite element arithmetic: it only draws random numbers
and evaluates closed-form fields at coordinates the caller supplies.  Both
sides call it with coordinates taken from their own meshes.

Workload recipes (all FP64, numpy ``default_rng``):

* manufactured solution u = sin(pi x) sin(pi y) sin(pi z) with
  f = -Laplace(u) = 3 pi^2 u (the plain Poisson problem of Section 3 of the
  paper, with the sin-product solution in place of the paper's tan/sin one);
* the paper's own manufactured pair (Section 2, Eqs. 2-3, a=1, b=2);
* a log-normal coefficient kappa = exp(g) per cell, g a Gaussian random field
  with squared-exponential covariance (sigma=1, length 0.2), realised by
  random Fourier features (Rahimi & Recht 2007) with M features;
* a smooth target u_d = sum of 8 seeded low-frequency sine products.
"""
import numpy as np

DEFAULT_SEED = 2104_08012


def rng(seed=DEFAULT_SEED):
    return np.random.default_rng(seed)


def sin_product(xyz):
    """u(x,y,z) = sin(pi x) sin(pi y) sin(pi z) at the rows of ``xyz`` (n,3)."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def sin_product_rhs(xyz):
    """f = -Laplace(sin product) = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)."""
    return 3.0 * np.pi ** 2 * sin_product(xyz)


def paper_solution(xyz, a=1.0, b=2.0):
    """The paper's analytic solution (Section 2, Eq. 3): sin(pi x) tan(pi x/4) sin(a pi y) sin(b pi z)."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    return np.sin(np.pi * x) * np.tan(np.pi * x / 4) * np.sin(a * np.pi * y) * np.sin(b * np.pi * z)


def paper_rhs(xyz, a=1.0, b=2.0):
    """The paper's right-hand side f (Section 2, Eq. 2), as printed."""
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    px = np.pi * x
    g = 2 * np.cos(px) - np.cos(px / 2) - 2 * (a * a + b * b) * np.sin(px) * np.tan(px / 4)
    return -np.pi ** 2 / 2 * g * np.sin(a * np.pi * y) * np.sin(b * np.pi * z)


def random_vector(n, seed=DEFAULT_SEED, dtype=np.float64):
    """Uniform(-1,1) test vector of length n."""
    return rng(seed).uniform(-1.0, 1.0, size=n).astype(dtype)


def grf_features(seed=DEFAULT_SEED, n_features=2048, length=0.2):
    """Frequencies omega ~ N(0, length^-2 I) and phases ~ U[0, 2 pi) of the RFF field."""
    r = rng(seed)
    omega = r.normal(0.0, 1.0 / length, size=(n_features, 3))
    phase = r.uniform(0.0, 2 * np.pi, size=n_features)
    return omega, phase


def grf_kappa(points, seed=DEFAULT_SEED, n_features=2048, length=0.2, sigma=1.0, chunk=1 << 16, device=None):
    """kappa = exp(g) at ``points`` (n,3), g = sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m).

    ``device``: optionally a torch device on which to evaluate the same FP64
    formula (for meshes of millions of cells; values agree with the numpy path
    to rounding).  Returns a numpy array either way.
    """
    omega, phase = grf_features(seed, n_features, length)
    scale = sigma * np.sqrt(2.0 / n_features)
    if device is not None:
        import torch
        om = torch.from_numpy(omega).to(device)
        ph = torch.from_numpy(phase).to(device)
        out = torch.empty(points.shape[0], dtype=torch.float64, device=device)
        for s in range(0, points.shape[0], chunk):
            p = torch.from_numpy(np.ascontiguousarray(points[s:s + chunk])).to(device)
            out[s:s + chunk] = scale * torch.cos(p @ om.T + ph).sum(dim=1)
        return torch.exp(out).cpu().numpy()
    out = np.empty(points.shape[0])
    for s in range(0, points.shape[0], chunk):
        p = points[s:s + chunk]
        out[s:s + chunk] = scale * np.cos(p @ omega.T + phase).sum(axis=1)
    return np.exp(out)


def target_field_params(seed=DEFAULT_SEED, n_terms=8):
    """Amplitudes a_m ~ N(0,1) and integer frequencies p,q,r in {1,2,3}."""
    r = rng(seed + 1)
    amp = r.normal(0.0, 1.0, size=n_terms)
    freq = r.integers(1, 4, size=(n_terms, 3))
    return amp, freq


def target_field(xyz, seed=DEFAULT_SEED, n_terms=8):
    """u_d = sum_m a_m sin(p_m pi x) sin(q_m pi y) sin(r_m pi z)."""
    amp, freq = target_field_params(seed, n_terms)
    out = np.zeros(xyz.shape[0])
    for a, (p, q, r) in zip(amp, freq):
        out += a * np.sin(p * np.pi * xyz[:, 0]) * np.sin(q * np.pi * xyz[:, 1]) * np.sin(r * np.pi * xyz[:, 2])
    return out


def batched_problem_table(seed=DEFAULT_SEED, n_problems=64, sizes=(16, 24, 32, 40, 48)):
    """Mesh sizes N_i drawn uniformly from ``sizes``; half P1 and half P2, interleaved by the seed.

    The default sizes are the multiples of 8 in [16, 48], so that every problem
    has a 4-level hierarchy whose coarse mesh has N_i/8 <= 6 cubes per axis.
    """
    r = rng(seed + 2)
    ns = r.choice(np.asarray(sizes), size=n_problems)
    degrees = np.array([1] * (n_problems // 2) + [2] * (n_problems - n_problems // 2))
    r.shuffle(degrees)
    return [(int(n), int(d)) for n, d in zip(ns, degrees)]
