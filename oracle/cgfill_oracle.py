"""FP64 CPU oracle: constrained Gaussian realizations on the flat torus.

TEST INFRASTRUCTURE ONLY -- used by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py``.  The product path never
imports it, and it shares no code with the CUDA path.

It follows Bucher & Louis, "Filling in CMB map missing data using constrained
Gaussian realizations" (arXiv:1109.0286):

* Sect. 2.1: pixels split into masked ``M`` (the paper's ``x``) and observed
  ``U`` (the paper's ``y``); ``C = P + N``; the maximum-likelihood fill is
  ``x_ML = -((C^-1)_MM)^-1 (C^-1)_MU d_U``.
* Sect. 2.3 (Hoffman-Ribak): draw an unconstrained ``y`` with covariance ``C``
  on the whole torus, then ``x_M = y_M + M (d - y)_U`` has the constrained
  covariance ``C_MM - C_MU C_UU^-1 C_UM`` (eq. starH).
* Sect. 2.4: solve ``(P_x C^-1 P_x) u = v`` (eq. ModEq) by conjugate gradients,
  optionally preconditioned by ``P_x C^{1/2} P_x`` on both sides.
* Sect. 4: on the torus the DFT is exactly unitary, so ``C^s`` is the
  diagonal ``P(k)^s`` in Fourier space.
* Sect. 5 (eqs. kern:rel, Boo, Algo): writing ``C^-1 = a (delta - K)`` with
  ``a`` the white high-k level of the precision, the ML fill satisfies
  ``x = K * x`` on M; iterating ``x_M <- (K * x)_M`` is the kernel relaxation.

DFT convention: ``F x(k) = sum_r x(r) exp(-i k.r)`` (unnormalised) and
``F^-1`` carries ``1/n``; ``C^s = F^-1 diag(P^s) F``.  The transform is the
oracle's own (``oracle_fft.c``: recursive mixed-radix decimation in time with
twiddles ``cos/sin(2 pi j/N)`` evaluated directly in FP64, rows and columns
split over host threads), pinned in the tests against a direct DFT.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
except the spectrum and mask recipes, which are input conventions.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import _native

__all__ = [
    "fft2", "ifft2", "fft_rows", "set_threads", "threads", "hermitian_full",
    "validate_spectrum", "apply_power", "philox4x32_10",
    "uniform52", "white_noise", "draw", "project", "rhs", "apply_A",
    "apply_S", "pcg", "PcgResult", "realize", "Realization",
    "dft2_direct", "circulant_corr", "dense_matrix", "ml_dense_cov",
    "ml_dense_prec", "constrained_cov_dense", "backward", "band_full",
    "relax_kernel", "relax", "disc_offsets", "subdivide", "strip_refine",
    "ms_radii", "annulus_offsets", "ms_classes", "laplace_ms",
    "loss_masked_sq", "lanczos_tridiag",
]


# ---------------------------------------------------------------------------
# The oracle's own DFT (Sect. 4: exactly unitary on the periodic grid)
# ---------------------------------------------------------------------------

_THREADS = max(1, int(os.cpu_count() or 1))


def set_threads(n: int) -> None:
    """Host threads of the transforms (the results do not depend on it)."""
    global _THREADS
    _THREADS = max(1, int(n))


def threads() -> int:
    return _THREADS


def _transform(x: np.ndarray, sign: int, rows_only: bool) -> np.ndarray:
    a = np.array(x, dtype=np.complex128, order="C", copy=True)
    if a.ndim != 2:
        raise ValueError("expected a 2-D array")
    fn = _native.lib().oracle_fft_rows if rows_only else _native.lib().oracle_fft2
    nthr = _THREADS if a.size >= 65536 else 1     # small maps: threads cost more than they save
    if fn(a.shape[0], a.shape[1], a.ctypes.data, sign, nthr) != 0:
        raise MemoryError("oracle FFT: out of host memory")
    return a


def fft2(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT ``X(k) = sum_r x(r) exp(-2 pi i (ky y/ny + kx x/nx))``."""
    return _transform(x, -1, False)


def ifft2(X: np.ndarray) -> np.ndarray:
    """Inverse 2D DFT, carrying the ``1/n``."""
    return _transform(X, +1, False) / (X.shape[0] * X.shape[1])


def fft_rows(x: np.ndarray) -> np.ndarray:
    """Unnormalised 1D DFT of every row of a 2-D array."""
    return _transform(x, -1, True)


# ---------------------------------------------------------------------------
# Spectrum on the torus (Sect. 4: F^dagger F = I on the periodic grid)
# ---------------------------------------------------------------------------

def hermitian_full(P_half: np.ndarray, nx: int) -> np.ndarray:
    """Extend a half-plane array ``ny x (nx/2+1)`` to the full ``ny x nx``
    plane using ``P(-k) = P(k)``."""
    ny = P_half.shape[0]
    full = np.empty((ny, nx), dtype=P_half.dtype)
    full[:, : nx // 2 + 1] = P_half
    my = (-np.arange(ny)) % ny
    for mx in range(nx // 2 + 1, nx):
        full[:, mx] = P_half[my, nx - mx]
    return full


def validate_spectrum(P_half: np.ndarray, nx: int) -> None:
    """P must be positive and finite, and real-symmetric on the two
    self-conjugate columns ``mx = 0`` and ``mx = nx/2`` (else ``C`` would
    not be a real symmetric operator)."""
    if not np.all(np.isfinite(P_half)) or np.any(P_half <= 0):
        raise ValueError("P(k) must be finite and > 0")
    my = (-np.arange(P_half.shape[0])) % P_half.shape[0]
    for col in (0, nx // 2):
        a, b = P_half[:, col], P_half[my, col]
        if np.any(np.abs(a - b) > 1e-12 * np.abs(a)):
            raise ValueError("P(k) is not Hermitian-consistent")


def apply_power(x: np.ndarray, P_full: np.ndarray, s: float) -> np.ndarray:
    """``C^s x = F^-1 diag(P^s) F x`` for a real map ``x``."""
    return np.real(ifft2(fft2(x) * P_full ** s))


# ---------------------------------------------------------------------------
# White noise: Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
# ---------------------------------------------------------------------------

_M32 = np.uint64(0xFFFFFFFF)
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words (held in uint64).

    One round: multiply words 0 and 2 by the two round multipliers, keep the
    high and low halves, and mix in words 1 and 3 and the key; between rounds
    the key is bumped by the two Weyl constants.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _M32 for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _M32
    k1 = np.asarray(k1, dtype=np.uint64) & _M32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _PHILOX_W0) & _M32
            k1 = (k1 + _PHILOX_W1) & _M32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniform52(a, b):
    """Uniform in (0, 1) from two 32-bit words: 52 random bits
    ``m = (a >> 6) * 2^26 + (b >> 6)``, value ``(m + 1/2) / 2^52`` (exact)."""
    m = (np.asarray(a, np.uint64) >> np.uint64(6)).astype(np.float64) * 67108864.0 \
        + (np.asarray(b, np.uint64) >> np.uint64(6)).astype(np.float64)
    return (m + 0.5) * (2.0 ** -52)


def white_noise(ny: int, nx: int, seed: int) -> np.ndarray:
    """Unit white noise xi(r) ~ N(0, 1) on the grid, fully set by ``seed``.

    Pixel pair ``j`` (row-major pixels ``2j`` and ``2j+1``) uses Philox counter
    ``(j, 0, 0, 0)`` and key ``(seed mod 2^32, seed >> 32)``; words (0, 1) and
    (2, 3) give two uniforms ``u1, u2``, and Box-Muller gives
    ``xi[2j] = sqrt(-2 ln u1) cos(2 pi u2)``, ``xi[2j+1] = ... sin(2 pi u2)``.
    """
    n = ny * nx
    j = np.arange(n // 2, dtype=np.uint64)
    zero = np.zeros_like(j)
    w0, w1, w2, w3 = philox4x32_10(j, zero, zero, zero,
                                   np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32))
    u1, u2 = uniform52(w0, w1), uniform52(w2, w3)
    rad = np.sqrt(-2.0 * np.log(u1))
    xi = np.empty(n, dtype=np.float64)
    xi[0::2] = rad * np.cos(2.0 * math.pi * u2)
    xi[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return xi.reshape(ny, nx)


def draw(P_full: np.ndarray, seed: int) -> np.ndarray:
    """Unconstrained realization with covariance C (Sect. 2.3, "easy because
    there are no cuts"): ``y = F^-1 [sqrt(P) F xi]``."""
    xi = white_noise(P_full.shape[0], P_full.shape[1], seed)
    return apply_power(xi, P_full, 0.5)


# ---------------------------------------------------------------------------
# Masked operator, right-hand side, preconditioner (Sects. 2.1, 2.4)
# ---------------------------------------------------------------------------

def project(v: np.ndarray, keep: np.ndarray) -> np.ndarray:
    """Projection ``P_x`` (or ``P_y``): zero every pixel outside ``keep``."""
    return np.where(keep, v, 0.0)


def rhs(P_full, observed, d, y):
    """``b = -(C^-1 z)_M`` with ``z = (d - y)`` on U and 0 on M
    (Sect. 2.1 with the Hoffman-Ribak substitution of Sect. 2.3)."""
    obs = observed.astype(bool)
    z = project(d - y, obs)
    return -project(apply_power(z, P_full, -1.0), ~obs)


def apply_A(v, P_full, masked):
    """``A v = P_x C^-1 P_x v`` (eq. ModEq)."""
    return project(apply_power(project(v, masked), P_full, -1.0), masked)


def apply_S(v, P_full, masked):
    """Preconditioner factor ``S v = P_x C^{1/2} P_x v`` (Sect. 2.4)."""
    return project(apply_power(project(v, masked), P_full, 0.5), masked)


@dataclass
class PcgResult:
    u: np.ndarray
    iters: int
    status: str                      # "converged" | "maxiter" | "breakdown"
    history: list = field(default_factory=list)   # ||r_k|| / ||b||, k = 0..iters
    alphas: list = field(default_factory=list)
    betas: list = field(default_factory=list)


def pcg(apply_a, b, apply_b=None, tol=1e-8, max_iter=10000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel, in the form
    reviewed by Golub & Van Loan, which the paper cites in Sect. 2.4).

    Solves ``A u = b`` from ``u = 0`` with preconditioner ``B ~ A^-1``
    (identity when ``apply_b`` is None) and stops when the recurrence residual
    satisfies ``||r|| <= tol ||b||``.  With ``B = S S`` this produces the same
    iterates as CG on the split system ``S A S u' = S b``, ``u = S u'``.
    """
    u = np.zeros_like(b)
    r = b.copy()
    bnorm = float(np.sqrt(np.sum(b * b)))
    res = PcgResult(u=u, iters=0, status="converged", history=[1.0 if bnorm > 0 else 0.0])
    if bnorm == 0.0:
        return res
    rho_old = None
    p = None
    k = 0
    while math.sqrt(float(np.sum(r * r))) > tol * bnorm:
        if k >= max_iter:
            res.status = "maxiter"
            break
        z = r if apply_b is None else apply_b(r)
        rho = float(np.sum(r * z))
        if k == 0:
            p = z.copy()
        else:
            beta = rho / rho_old
            res.betas.append(beta)
            p = z + beta * p
        q = apply_a(p)
        pq = float(np.sum(p * q))
        if not (pq > 0.0) or not (rho > 0.0):
            res.status = "breakdown"
            break
        alpha = rho / pq
        res.alphas.append(alpha)
        u = u + alpha * p
        r = r - alpha * q
        rho_old = rho
        k += 1
        res.history.append(math.sqrt(float(np.sum(r * r))) / bnorm)
    res.u, res.iters = u, k
    return res


@dataclass
class Realization:
    x: np.ndarray          # the constrained realization (x_U = d_U exactly)
    y: np.ndarray          # the unconstrained draw
    u: np.ndarray          # the ML correction on M (0 on U)
    b: np.ndarray          # the right-hand side on M (0 on U)
    pcg: PcgResult
    true_rel_resid: float


def realize(P_half, observed, d, seed, tol=1e-8, precond=True, max_iter=10000):
    """One constrained Gaussian realization (Sects. 2.1-2.4).

    ``y = F^-1 sqrt(P) F xi(seed)``; solve ``A u = b`` with
    ``b = -(C^-1 (d - y)_U)_M``; return ``x_M = y_M + u`` and ``x_U = d_U``.
    """
    ny, nx = observed.shape
    validate_spectrum(P_half, nx)
    P_full = hermitian_full(P_half, nx)
    obs = observed.astype(bool)
    masked = ~obs
    d = np.asarray(d, dtype=np.float64)
    y = draw(P_full, seed)
    b = rhs(P_full, observed, d, y)
    A = lambda v: apply_A(v, P_full, masked)          # noqa: E731
    B = (lambda v: apply_S(apply_S(v, P_full, masked), P_full, masked)) if precond else None  # noqa: E731
    res = pcg(A, b, B, tol=tol, max_iter=max_iter)
    x = np.where(obs, d, y + res.u)
    bn = math.sqrt(float(np.sum(b * b)))
    tr = b - A(res.u)
    true_rel = math.sqrt(float(np.sum(tr * tr))) / bn if bn > 0 else 0.0
    return Realization(x=x, y=y, u=res.u, b=b, pcg=res, true_rel_resid=true_rel)


# ---------------------------------------------------------------------------
# Dense brute force (Sect. 6.5 validates against a direct solve)
# ---------------------------------------------------------------------------

def dft2_direct(x: np.ndarray) -> np.ndarray:
    """Unnormalised 2D DFT by its definition, as two dense matrix products."""
    ny, nx = x.shape
    Ey = np.exp(-2j * math.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    Ex = np.exp(-2j * math.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    return Ey @ x @ Ex.T


def circulant_corr(P_full: np.ndarray, s: float = 1.0) -> np.ndarray:
    """``c(D) = (1/n) sum_k P(k)^s cos(k.D)``: the torus correlation of
    ``C^s`` at every displacement D, from the definition (no FFT)."""
    ny, nx = P_full.shape
    Ey = np.exp(2j * math.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    Ex = np.exp(2j * math.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    return np.real(Ey @ (P_full ** s) @ Ex.T) / (ny * nx)


def dense_matrix(corr: np.ndarray, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Block ``[C]_{ij} = c(r_i - r_j)`` for flat pixel indices ``rows, cols``."""
    ny, nx = corr.shape
    yi, xi = np.divmod(rows, nx)
    yj, xj = np.divmod(cols, nx)
    return corr[(yi[:, None] - yj[None, :]) % ny, (xi[:, None] - xj[None, :]) % nx]


def ml_dense_cov(P_full, observed, dU):
    """``x_ML = C_MU C_UU^-1 d_U`` by Cholesky (the covariance form)."""
    obs = observed.ravel().astype(bool)
    M, U = np.nonzero(~obs)[0], np.nonzero(obs)[0]
    c = circulant_corr(P_full, 1.0)
    L = np.linalg.cholesky(dense_matrix(c, U, U))
    t = np.linalg.solve(L.T, np.linalg.solve(L, dU))
    return dense_matrix(c, M, U) @ t


def ml_dense_prec(P_full, observed, dU):
    """``x_ML = -((C^-1)_MM)^-1 (C^-1)_MU d_U`` (Sect. 2.1, precision form)."""
    obs = observed.ravel().astype(bool)
    M, U = np.nonzero(~obs)[0], np.nonzero(obs)[0]
    q = circulant_corr(P_full, -1.0)
    return -np.linalg.solve(dense_matrix(q, M, M), dense_matrix(q, M, U) @ dU)


def constrained_cov_dense(P_full, observed):
    """``C_MM - C_MU C_UU^-1 C_UM`` (eq. starH)."""
    obs = observed.ravel().astype(bool)
    M, U = np.nonzero(~obs)[0], np.nonzero(obs)[0]
    c = circulant_corr(P_full, 1.0)
    CUU = dense_matrix(c, U, U)
    CMU = dense_matrix(c, M, U)
    return dense_matrix(c, M, M) - CMU @ np.linalg.solve(CUU, CMU.T)


# ---------------------------------------------------------------------------
# Gradient of L = sum_M x^2 through the realization (adjoint method)
# ---------------------------------------------------------------------------

def loss_masked_sq(x, observed):
    """``L = sum_{i in M} x_i^2``."""
    return float(np.sum(np.where(observed.astype(bool), 0.0, x) ** 2))


def band_full(bidx_half: np.ndarray, nx: int) -> np.ndarray:
    """Band index of every full-plane mode (Hermitian extension)."""
    return hermitian_full(bidx_half, nx)


def backward(P_half, observed, d, seed, real: Realization, bidx_half, sig_half,
             tol=1e-8, precond=True, max_iter=10000):
    """Gradients of ``L = sum_M x^2`` w.r.t. the data ``d`` and the band
    amplitudes ``a_b`` of ``P(k) = sum_b a_b 1[k in b] S(k) + N``.

    With ``w = (d - y)`` on U and ``u`` on M (so ``(C^-1 w)_M = 0``),
    ``g = 2 x_M`` and the adjoint ``lam = A^-1 g`` (one more solve with the
    same symmetric operator):

    * ``dL/dd_U = -(C^-1 lam)_U`` and ``dL/dd_M = 0``;
    * ``h = g`` on M and ``(C^-1 lam)_U`` on U is ``dL/dy``;
    * ``dL/dP(k) = Re[conj(F h) F xi] / (2 n sqrt(P))
      + Re[conj(F lam) F w] / (n P^2)`` per full-plane mode, and
      ``dL/da_b = sum_k 1[k in b] S(k) dL/dP(k)``.

    The noise draw ``xi`` is held fixed by the seed (a reparameterised
    gradient).  Returns ``(grad_d, grad_bands, lam)``.
    """
    ny, nx = observed.shape
    P_full = hermitian_full(P_half, nx)
    obs = observed.astype(bool)
    masked = ~obs
    n = ny * nx
    g = np.where(masked, 2.0 * real.x, 0.0)
    A = lambda v: apply_A(v, P_full, masked)          # noqa: E731
    B = (lambda v: apply_S(apply_S(v, P_full, masked), P_full, masked)) if precond else None  # noqa: E731
    lam = pcg(A, g, B, tol=tol, max_iter=max_iter).u
    Qlam = apply_power(lam, P_full, -1.0)
    grad_d = np.where(obs, -Qlam, 0.0)
    h = np.where(masked, g, Qlam)
    w = np.where(obs, d - real.y, real.u)
    xi_hat = fft2(white_noise(ny, nx, seed))
    dLdP = (np.real(np.conj(fft2(h)) * xi_hat) / (2.0 * n * np.sqrt(P_full))
            + np.real(np.conj(fft2(lam)) * fft2(w)) / (n * P_full ** 2))
    bfull = band_full(bidx_half, nx)
    sfull = hermitian_full(sig_half, nx)
    nb = int(bidx_half.max()) + 1
    grad_b = np.bincount(bfull.ravel(), weights=(sfull * dLdP).ravel(), minlength=nb)
    return grad_d, grad_b, lam


# ---------------------------------------------------------------------------
# Lanczos tridiagonal from the CG coefficients (Sect. 6.4 uses Lanczos for
# the condition number)
# ---------------------------------------------------------------------------

def lanczos_tridiag(alphas, betas):
    """Tridiagonal Lanczos matrix of the preconditioned operator built from
    CG's step lengths ``alpha_j`` and direction updates ``beta_j``:
    ``T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}``,
    ``T_{j,j+1} = sqrt(beta_j)/alpha_j``."""
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    return T


# ---------------------------------------------------------------------------
# Kernel relaxation (Sect. 5, eqs. kern:rel, Boo and Algo) on the torus
# ---------------------------------------------------------------------------

def relax_kernel(P_full):
    """``(a, K)`` with ``C^-1 = a (delta - K)`` as in eq. kern:rel: ``a`` is the
    white (high-k) level of the precision, ``a = max_k 1/P(k)`` (for
    ``P = S + N`` with white noise N, ``a = 1/N`` once the signal has died
    off), so that ``K^(k) = 1 - 1/(a P(k))`` lies in [0, 1) and the convolution
    with K is a weighted average (the singular part of C^-1 is the delta term,
    the smooth regular part -a K).  K at every displacement comes from the
    correlation function of C^-1 (no FFT)."""
    q = circulant_corr(P_full, -1.0)
    a = float(np.max(1.0 / P_full))
    K = -q / a
    K[0, 0] += 1.0
    return a, K


def relax(P_half, observed, d, iters):
    """Kernel relaxation, eq. Algo: from ``x_M = 0`` and ``x_U = d_U``, repeat
    ``x_M <- (K * x)_M`` with the kernel of ``relax_kernel``, i.e.
    ``x_M <- x_M - (C^-1 x)_M / a``.  Its fixed point solves ``(C^-1 x)_M = 0``
    (eq. Boo: the ML fill), and since ``0 < C^-1/a <= 1`` it contracts.
    Returns the map and ``||(C^-1 x)_M||`` before each step."""
    ny, nx = observed.shape
    P_full = hermitian_full(P_half, nx)
    obs = observed.astype(bool)
    a = float(np.max(1.0 / P_full))
    x = project(np.asarray(d, dtype=np.float64), obs)
    norms = []
    for _ in range(iters):
        v = apply_power(x, P_full, -1.0)
        norms.append(float(np.linalg.norm(v[~obs])))
        x[~obs] -= v[~obs] / a
    return x, norms


# ---------------------------------------------------------------------------
# Subdivision of the mask (Sect. 6.2) and strip refinement (Sect. 6.4)
# ---------------------------------------------------------------------------

def disc_offsets(radius):
    """Lattice offsets ``(dy, dx)`` with ``dy^2 + dx^2 <= radius^2``."""
    R = int(math.floor(radius))
    return [(dy, dx) for dy in range(-R, R + 1) for dx in range(-R, R + 1)
            if dy * dy + dx * dx <= radius * radius]


def subdivide(observed, delta, threshold=0.03):
    """Sect. 6.2: the boundary layer of width ``delta``: convolve the observed
    indicator (1 on U, 0 on M) with the normalised top hat of radius
    ``delta / 2`` (periodic) and keep the masked pixels whose value exceeds
    ``threshold``.  The convolution is a pixel count over the disc, computed
    here by FFT and rounded to the integer it equals; the comparison
    ``count > threshold * |disc|`` is then exact.  Returns a bool map."""
    ny, nx = observed.shape
    offs = disc_offsets(delta / 2.0)
    disc = np.zeros((ny, nx))
    for dy, dx in offs:
        disc[dy % ny, dx % nx] = 1.0
    obs = observed.astype(bool)
    count = np.rint(np.real(ifft2(fft2(obs.astype(np.float64)) * fft2(disc)))).astype(np.int64)
    return (~obs) & (count * 100 > round(threshold * 100) * len(offs))


def strip_refine(S_half, N_half, observed, d, stages, tol=1e-8, max_iter=10000, x0=None):
    """Sect. 6.4 on the torus: for each ``(beta, w)`` in turn, the strip
    ``D = subdivide(observed, w)`` of the original mask is refilled with the
    maximum-likelihood solution for the boosted-noise spectrum
    ``P = S + beta N``, the current map outside the strip acting as data
    (PCG with the sqrt(C) preconditioner to ``tol``).  Starts from ``x0`` on
    the mask (default 0); ``d`` on U is never changed.  Returns the map."""
    ny, nx = observed.shape
    obs = observed.astype(bool)
    x = np.where(obs, np.asarray(d, dtype=np.float64), 0.0 if x0 is None else x0)
    for beta, w in stages:
        strip = subdivide(observed, w)
        if not strip.any():
            continue
        P_full = hermitian_full(S_half + beta * N_half, nx)
        b = rhs(P_full, (~strip).astype(np.uint8), x, np.zeros_like(x))
        res = pcg(lambda v: apply_A(v, P_full, strip), b,
                  lambda v: apply_S(apply_S(v, P_full, strip), P_full, strip),
                  tol=tol, max_iter=max_iter)
        x = np.where(strip, res.u, x)
    return x


# ---------------------------------------------------------------------------
# Multi-scale kernel Laplace solver (Sect. 6.3) on the torus
# ---------------------------------------------------------------------------

def ms_radii(nk=9, rho0=1.5, q=1.55):
    """``nk`` annuli ``(r_in, r_out)`` with centre radii ``rho_j = rho0 q^j`` in
    geometric progression and bounds at the geometric midpoints
    ``rho_j / sqrt(q)``, ``rho_j sqrt(q)``, so consecutive annuli tile the
    plane; the smallest is solid (``r_in = 0``, centre pixel excluded)."""
    out = []
    for j in range(nk):
        rho = rho0 * q ** j
        out.append((0.0 if j == 0 else rho / math.sqrt(q), rho * math.sqrt(q)))
    return out


def annulus_offsets(r_in, r_out):
    """Lattice offsets with ``r_in^2 < dy^2 + dx^2 <= r_out^2`` (never the centre)."""
    R = int(math.floor(r_out))
    return [(dy, dx) for dy in range(-R, R + 1) for dx in range(-R, R + 1)
            if max(r_in * r_in, 0.0) < dy * dy + dx * dx <= r_out * r_out and (dy or dx)]


def ms_classes(observed, radii):
    """Kernel index of every masked pixel: the largest ``j`` whose disc of
    radius ``r_out_j`` around the pixel holds no observed pixel, else 0 (the
    thin boundary layer, where the smallest kernel reaches the observed
    region and carries its values in).  Observed pixels get 0."""
    obs = observed.astype(bool)
    cls = np.zeros(observed.shape, dtype=np.int64)
    for j, (_, r_out) in enumerate(radii):
        inside = (~obs) & ~subdivide(observed, 2.0 * r_out, 0.0)
        cls[inside] = j
    return cls


def laplace_ms(observed, d, radii, iters):
    """Sect. 6.3 on the torus: from 0 on the mask and ``d`` on the observed
    pixels, every sweep replaces each masked value by the average of the
    previous map over its class's annulus (Jacobi: all averages from the same
    map), by FFT convolution with the normalised annulus.  Returns the map."""
    ny, nx = observed.shape
    obs = observed.astype(bool)
    cls = ms_classes(observed, radii)
    spectra = []
    for r_in, r_out in radii:
        k = np.zeros((ny, nx))
        offs = annulus_offsets(r_in, r_out)
        for dy, dx in offs:
            k[dy % ny, dx % nx] = 1.0 / len(offs)
        spectra.append(fft2(k))
    x = np.where(obs, np.asarray(d, dtype=np.float64), 0.0)
    for _ in range(iters):
        X = fft2(x)
        new = x.copy()
        for j, K in enumerate(spectra):
            sel = (~obs) & (cls == j)
            if sel.any():
                new[sel] = np.real(ifft2(X * K))[sel]
        x = new
    return x
