"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and scales them; it contains none of
the method's arithmetic, so the tests may feed the same inputs to the CUDA
library and to the CPU oracle.  Each generator documents its recipe.

The paper uses randn matrices (Sec. 5: A = randn(100)), a Toeplitz matrix
A_ij = 1/(1+(i-j)^2) (Eq. Ex2b) and trid{-1,2,-1} (Sec. 5); the batched and
large shapes below stand in for those experiments at production sizes.
"""
import numpy as np


def _rng(seed):
    return np.random.default_rng(seed)


def dense_scaled(d, norm1, seed, scale_sqrt=False):
    """N(0,1) entries (divided by sqrt(d) if scale_sqrt), then scaled so that
    ||A||_1 = norm1 exactly up to rounding."""
    g = _rng(seed)
    A = g.standard_normal((d, d))
    if scale_sqrt:
        A /= np.sqrt(d)
    return A * (norm1 / np.abs(A).sum(axis=0).max())


def single_d64(seed=0):
    """One real d = 64 matrix, N(0,1) scaled to ||A||_1 = 2, and v ~ N(0,1)."""
    A = dense_scaled(64, 2.0, seed)
    v = _rng(seed + 1).standard_normal(64)
    return A, v


def batch_dims(batch, seed, choices=tuple(range(16, 257, 16))):
    """d_b drawn uniformly from choices (default {16, 32, ..., 256})."""
    return _rng(seed).choice(np.array(choices), size=batch)


def batch_mixed_d(batch=4096, seed=1000, choices=tuple(range(16, 257, 16)), lo=0.5, hi=8.0):
    """Batch of real dense matrices: d uniform over choices; entries
    N(0,1)/sqrt(d); each scaled to ||A||_1 ~ U[lo, hi].  Returns (dims, list of
    matrices, norms).  Matrix b uses seed + 1 + b."""
    dims = batch_dims(batch, seed, choices)
    norms = _rng(seed + 7919).uniform(lo, hi, size=batch)
    mats = [dense_scaled(int(d), float(n), seed + 1 + b, scale_sqrt=True)
            for b, (d, n) in enumerate(zip(dims, norms))]
    return dims, mats, norms


def batch_flat(dims, norms, seed=1000):
    """The same batch as batch_mixed_d, packed back to back (float64)."""
    out = np.empty(int(np.sum(np.asarray(dims, dtype=np.int64) ** 2)))
    o = 0
    for b, (d, n) in enumerate(zip(dims, norms)):
        d = int(d)
        out[o:o + d * d] = dense_scaled(d, float(n), seed + 1 + b, scale_sqrt=True).ravel()
        o += d * d
    return out


def hermitian_parts(d=4096, m=256, seed=2000):
    """H = (G + G^H)/2 with G complex N(0,1)/sqrt(d), and V complex N(0,1), d x m,
    before any scaling (the same draws on every machine)."""
    g = _rng(seed)
    G = (g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))) / np.sqrt(d)
    H = (G + G.conj().T) / 2
    V = g.standard_normal((d, m)) + 1j * g.standard_normal((d, m))
    return H, V


def hermitian_scale(H, rho):
    """The factor that gives H spectral radius rho (an eigenvalue routine: its
    last bits may differ between machines)."""
    return rho / np.abs(np.linalg.eigvalsh(H)).max()


def hermitian_action(d=4096, m=256, rho=20.0, seed=2000, scale=None):
    """A = -iH, H = (G + G^H)/2 with G complex N(0,1)/sqrt(d), scaled so that its
    spectral radius is rho (or by the given scale, which rebuilds the same A
    bit for bit); V complex N(0,1), d x m.  Returns (A, V, rho)."""
    H, V = hermitian_parts(d, m, seed)
    if scale is None:
        scale = hermitian_scale(H, rho)
    H *= scale
    return -1j * H, V, rho


def diffusion_batch(batch=512, d=512, seed=3000, tmin=1e-4, tmax=1e-2):
    """A_b = -L + 0.1 N_b, L = trid{-1, 2, -1} / h^2 with h = 1/(d+1), N_b with
    N(0,1)/sqrt(d) entries; t_b log-uniform in [tmin, tmax]; u0_b, b_b ~ N(0,1)."""
    h = 1.0 / (d + 1)
    L = (np.diag(np.full(d, 2.0)) - np.diag(np.ones(d - 1), 1) - np.diag(np.ones(d - 1), -1)) / h ** 2
    g = _rng(seed)
    mats = [-L + 0.1 * g.standard_normal((d, d)) / np.sqrt(d) for _ in range(batch)]
    ts = np.exp(g.uniform(np.log(tmin), np.log(tmax), size=batch))
    u0 = g.standard_normal((batch, d))
    bb = g.standard_normal((batch, d))
    return mats, ts, u0, bb


def grad_batch(batch=256, d=128, seed=4000):
    """A_b with N(0,1)/sqrt(d) entries; v_b, y_b ~ N(0,1)."""
    g = _rng(seed)
    A = g.standard_normal((batch, d, d)) / np.sqrt(d)
    v = g.standard_normal((batch, d))
    y = g.standard_normal((batch, d))
    return A, v, y


def toeplitz_paper(d=100):
    """Eq. (Ex2b): A_ij = 1/(1 + (i - j)^2)."""
    i = np.arange(d)
    return 1.0 / (1.0 + (i[:, None] - i[None, :]) ** 2)


def trid_batch(batch, d, eta=8.0, seed=5000, spread=0.1):
    """A batch of tridiagonal systems shaped like the paper's trid{-1,2,-1}
    example (Sec. 5, Fig. 4, d = 1000), negated so that exp(tA) decays as in a
    diffusion step: A_b = -trid{1 + e', 2 (1 + e), 1 + e''} with e, e', e''
    ~ spread N(0,1) / 2 per entry; v_b = w / ||w||_2, w ~ N(0,1) (the paper's
    unit random vector); t_b = eta / ||A_b||_1, so ||t_b A_b||_1 = eta up to
    rounding.  Returned batch-interleaved, shape (d, batch): row k holds entry
    k of every system (dl[0] and du[d-1] are zero and not part of A)."""
    g = _rng(seed)
    h = spread / 2
    dd = -2.0 * (1.0 + h * g.standard_normal((d, batch)))
    dl = 1.0 + h * g.standard_normal((d, batch))
    du = 1.0 + h * g.standard_normal((d, batch))
    dl[0] = 0.0
    du[d - 1] = 0.0
    w = g.standard_normal((d, batch))
    v = w / np.linalg.norm(w, axis=0)
    # ||A_b||_1: column k holds du[k-1], dd[k], dl[k+1]
    col = np.abs(dd).copy()
    col[1:] += np.abs(du[:-1])
    col[:-1] += np.abs(dl[1:])
    t = eta / col.max(axis=0)
    return dl, dd, du, v, t


def trid_dense(dl, dd, du, b):
    """System b of a batch-interleaved tridiagonal batch as a dense matrix."""
    d = dd.shape[0]
    A = np.diag(dd[:, b])
    if d > 1:
        A += np.diag(dl[1:, b], -1) + np.diag(du[:-1, b], 1)
    return A


def penta_batch(batch, d, eta=8.0, seed=6000, spread=0.1):
    """A batch of pentadiagonal systems: the fourth-order central stencil of the
    second derivative, (-1, 16, -30, 16, -1) / 12 (so exp(tA) decays as in a
    diffusion step), each entry perturbed by a factor 1 + spread N(0,1)/2;
    v_b = w / ||w||_2, w ~ N(0,1); t_b = eta / ||A_b||_1.  Returned as diags of
    shape (5, d, batch), diags[j, k, b] = A_b[k][k + j - 2] (zero outside the
    matrix), and v, t."""
    g = _rng(seed)
    h = spread / 2
    stencil = np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0
    diags = stencil[:, None, None] * (1.0 + h * g.standard_normal((5, d, batch)))
    for j in range(5):
        o = j - 2
        for k in range(d):
            if not 0 <= k + o < d:
                diags[j, k, :] = 0.0
    w = g.standard_normal((d, batch))
    v = w / np.linalg.norm(w, axis=0)
    col = np.zeros((d, batch))
    for j in range(5):  # column k + o gets |A[k][k + o]|
        o = j - 2
        for k in range(d):
            if 0 <= k + o < d:
                col[k + o] += np.abs(diags[j, k])
    t = eta / col.max(axis=0)
    return diags, v, t


def band_dense(diags, b):
    """System b of a batch-interleaved banded batch (diags (2p+1, d, batch)) as a
    dense matrix."""
    q, d, _ = diags.shape
    p = (q - 1) // 2
    A = np.zeros((d, d))
    for j in range(q):
        o = j - p
        for k in range(d):
            if 0 <= k + o < d:
                A[k, k + o] = diags[j, k, b]
    return A
