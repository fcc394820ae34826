"""Seeded synthetic inputs for the CCM workloads (numpy, float64 then float32).

This module holds no part of the method's arithmetic: it only makes series.
Both the oracle tests and the CUDA tests/bench draw their inputs from here.

Every generator simulates in float64, z-normalises each series (population
standard deviation) and casts once to float32; the float32 values are what
both the GPU path and the oracle read.

Workloads (shapes and distributions of the paper's use cases; the paper's own
datasets are not available, these stand in for them):
  coupled logistic maps  x_i(t+1) = x_i(t) (r_i - r_i x_i(t) - sum_j b_ij x_j(t))
  calcium-imaging-like   exp-filtered projections of a shared Lorenz-63 driver
                         plus independent AR(1) noise.
"""
import math

import numpy as np

# Rows of the coupling matrix whose sum exceeds this are scaled down to it.
# With sum_j b_ij <= 0.09 and x in (0, r/4], the bracket r(1-x) - sum b x stays
# positive for every r >= 3.6 (min over r of r(1 - r/4) = 0.0975 > 0.09 * 0.975),
# so the maps stay in (0, 1) and never diverge.
BETA_ROW_CAP = 0.09


def znorm32(X):
    """z-normalise each row in float64 (population std), cast to float32."""
    X = np.asarray(X, np.float64)
    mu = X.mean(axis=-1, keepdims=True)
    sd = X.std(axis=-1, keepdims=True)
    sd[sd == 0] = 1.0
    return np.ascontiguousarray(((X - mu) / sd).astype(np.float32))


def coupled_logistic(N, L, seed, r_lo=3.7, r_hi=3.9, p_beta=0.2, beta_max=0.05,
                     noise=0.0, burn=500, return_info=False):
    """N coupled logistic maps of length L, z-normalised float32 [N][L].

    r_i ~ U[r_lo, r_hi], b_ij != 0 with probability p_beta (b_ii = 0) and value
    U[0, beta_max], x_i(0) ~ U[0.2, 0.8], `burn` steps discarded, then optional
    Gaussian observation noise of std `noise` before normalisation.
    """
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_lo, r_hi, N)
    mask = rng.random((N, N)) < p_beta
    beta = np.where(mask, rng.uniform(0.0, beta_max, (N, N)), 0.0)
    np.fill_diagonal(beta, 0.0)
    rows = beta.sum(axis=1)
    over = rows > BETA_ROW_CAP
    beta[over] *= (BETA_ROW_CAP / rows[over])[:, None]
    x = rng.uniform(0.2, 0.8, N)
    use_sparse = N > 256
    if use_sparse:
        import scipy.sparse as sp
        B = sp.csr_matrix(beta)
    else:
        B = beta
    out = np.empty((N, L), np.float64)
    for t in range(burn + L):
        x = x * (r - r * x - B @ x)
        if t >= burn:
            out[:, t - burn] = x
    if not np.all(np.isfinite(out)):
        raise FloatingPointError("coupled logistic diverged")
    if noise > 0:
        out += rng.normal(0.0, noise, out.shape)
    X = znorm32(out)
    if return_info:
        return X, {"beta": beta, "r": r, "beta_rows_rescaled": int(over.sum())}
    return X


def lorenz63(n_samples, seed, dt=0.01, every=5, burn=1000, sigma=10.0,
             rho=28.0, beta=8.0 / 3.0):
    """Lorenz-63 by RK4 (step dt), one sample every `every` steps, `burn`
    samples discarded; each component standardised.  Returns [n_samples][3]."""
    rng = np.random.default_rng(seed)
    s = np.array([1.0, 1.0, 1.0]) + rng.normal(0.0, 0.1, 3)

    def f(v):
        return np.array([sigma * (v[1] - v[0]),
                         v[0] * (rho - v[2]) - v[1],
                         v[0] * v[1] - beta * v[2]])

    out = np.empty((n_samples, 3))
    for i in range(burn + n_samples):
        for _ in range(every):
            k1 = f(s)
            k2 = f(s + 0.5 * dt * k1)
            k3 = f(s + 0.5 * dt * k2)
            k4 = f(s + dt * k3)
            s = s + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if i >= burn:
            out[i - burn] = s
    out -= out.mean(axis=0)
    out /= out.std(axis=0)
    return out


def calcium_lorenz(N, L, seed, tau_decay=5.0, phi=0.9, ar_sigma=0.5,
                   filt_burn=50):
    """Calcium-imaging-shaped series, z-normalised float32 [N][L].

    series_i = exp-filter(alpha = exp(-1/tau_decay)) of (W_i . z(t) + a_i(t)),
    z a standardised Lorenz-63 driver shared by all series, W_i ~ N(0,1)^3 and
    a_i an AR(1) process with coefficient phi and innovation std ar_sigma.
    """
    rng = np.random.default_rng(seed)
    T = L + filt_burn
    z = lorenz63(T, seed + 7919)
    W = rng.normal(0.0, 1.0, (N, 3))
    alpha = math.exp(-1.0 / tau_decay)
    a = rng.normal(0.0, ar_sigma / math.sqrt(1.0 - phi * phi), N)
    c = None
    out = np.empty((N, L), np.float64)
    for t in range(T):
        a = phi * a + rng.normal(0.0, ar_sigma, N)
        s = W @ z[t] + a
        c = s if c is None else alpha * c + (1.0 - alpha) * s
        if t >= filt_burn:
            out[:, t - filt_burn] = c
    return znorm32(out)


# --- the five workload recipes ------------------------------------------------

def logistic_16x200():
    """16 coupled-logistic series, L=200 (r~U[3.7,3.9], 20% b~U[0,0.05])."""
    return coupled_logistic(16, 200, 1001, 3.7, 3.9, 0.2, 0.05)


def logistic_noisy(N=1000, L=1000):
    """1,000 x 1,000 coupled logistic, r~U[3.6,3.9], 5% b~U[0,0.1], noise 0.01."""
    return coupled_logistic(N, L, 1002, 3.6, 3.9, 0.05, 0.1, noise=0.01)


def calcium(N=50000, L=1500, seed=1003):
    """Calcium-imaging-shaped all-to-all workload, 50,000 x 1,500."""
    return calcium_lorenz(N, L, seed)


def uneven_batch_shapes(n_inst=256, seed=1004):
    """(N, L) of the uneven batch: log-uniform ints N in [32, 2048],
    L in [200, 5000]."""
    rng = np.random.default_rng(seed)
    N = np.exp(rng.uniform(math.log(32), math.log(2048 + 1), n_inst)).astype(int)
    L = np.exp(rng.uniform(math.log(200), math.log(5000 + 1), n_inst)).astype(int)
    return np.minimum(N, 2048), np.minimum(L, 5000)


def uneven_batch_instance(i, N, L, seed=1004):
    return coupled_logistic(int(N), int(L), seed * 1000 + i, 3.6, 3.9, 0.05, 0.1,
                            noise=0.02)


def logistic_long(N=2000, L=10000):
    """2,000 x 10,000 coupled logistic for the library-length sweep."""
    return coupled_logistic(N, L, 1005, 3.6, 3.9, 0.05, 0.1, noise=0.01)


def logistic_map(L, r=3.8, x0=0.4, burn=100):
    """Noise-free single logistic map, float32 (not normalised)."""
    x = x0
    out = np.empty(L)
    for t in range(burn + L):
        x = r * x * (1.0 - x)
        if t >= burn:
            out[t - burn] = x
    return out.astype(np.float32)


def logistic_pair(L, seed, r_x=3.8, r_y=3.5, b_xy=0.0, b_yx=0.1, burn=200):
    """Two coupled logistic maps (x drives y when b_yx > 0, b_xy = 0):
    x(t+1) = x(t)(r_x - r_x x(t) - b_xy y(t)),
    y(t+1) = y(t)(r_y - r_y y(t) - b_yx x(t)).  float32 [2][L], z-normalised."""
    rng = np.random.default_rng(seed)
    x, y = rng.uniform(0.2, 0.8, 2)
    out = np.empty((2, L))
    for t in range(burn + L):
        x, y = x * (r_x - r_x * x - b_xy * y), y * (r_y - r_y * y - b_yx * x)
        if t >= burn:
            out[:, t - burn] = (x, y)
    return znorm32(out)


def ar1_series(N, L, seed, phi=0.9, sigma=1.0, burn=50):
    """N independent AR(1) series x(t+1) = phi x(t) + sigma e(t), float32
    [N][L], generated a time step at a time (cheap for very many series);
    stands in for the 10^5 targets x 10^4 steps of the paper's lookup
    micro-benchmark."""
    rng = np.random.default_rng(seed)
    out_t = np.empty((L, N), np.float32)  # time-major while generating
    x = rng.standard_normal(N, dtype=np.float32)
    phi32, sig32 = np.float32(phi), np.float32(sigma)
    for t in range(burn + L):
        x = phi32 * x + sig32 * rng.standard_normal(N, dtype=np.float32)
        if t >= burn:
            out_t[t - burn] = x
    return np.ascontiguousarray(out_t.T)
