"""CPU FP64 oracle for ChASE's hot path -- TEST INFRASTRUCTURE, not product code.

This module is a plain, slow, step-by-step NumPy restatement of the ChASE
algorithms (Winkelmann, Springer, Di Napoli, "ChASE: Chebyshev Accelerated
Subspace iteration Eigensolver for sequences of Hermitian eigenvalue
problems", arXiv 1805.10121).  Every function names the algorithm, equation
or section it follows.  Arithmetic is complex128 / float64 throughout.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference arm) may import it.  It shares no code with the CUDA
library: matrix products use NumPy's ``@`` (a library primitive), while the
QR factorisation, the Hermitian eigensolver, the Lanczos process, the
spectral-density estimate, the degree rule and the locking rule are written
out here.

Readings of the paper where it is silent or ambiguous (each is listed in the
design notes as well):

* Residual test: ``conv_mode="abs"`` locks at ``Res <= tol`` (Sec. 6.1 says
  ChASE uses an absolute criterion); ``conv_mode="rel"`` locks at
  ``Res <= tol * h`` with ``h`` the largest ``|theta|`` over every Ritz value
  seen so far (Lanczos and Rayleigh-Ritz).  Since ``|theta| <= ||H||_2`` this
  implies ``Res <= tol * ||H||_2``.  The degree rule (Alg. 5) uses the same
  effective tolerance.
* Alg. 1 line 7 passes the whole basis to RAYLEIGH-RITZ; the loop keeps the
  locked vectors fixed, so RR runs on the active columns only (the ``RR(ritzv,
  block)`` kernel of Listing 1 does the same).
* Alg. 1 line 13 uses the Ritz value of the active column.
* Alg. 5 when ``|rho| <= 1`` (Ritz value inside the damped interval) or the
  quotient is not finite: the degree is DEGMAX.  The even rounding of line 6
  is applied after the DEGMAX clamp; an odd DEGMAX is then lowered by one.
* The initial degree ``deg`` of Alg. 1 line 1 is rounded up to even.
* Sorts are stable: by Ritz value (Alg. 3 line 2), then by degree (Alg. 1
  line 15).
* Lanczos (Alg. 6): no re-orthogonalisation.  When ``approx`` is false the
  upper bound is the largest ``||f_k|| + max theta`` over the first run and all
  ``n_vec`` density runs.  The Gaussian width ``sigma`` is measured in the
  variable that maps ``[mu_1, b_sup]`` onto ``[-1, 1]``.  The Eq. 10 sum runs
  over the ``k`` Ritz values of each run.  If the quantile of line 11 is not
  strictly inside ``(mu_1, b_sup)`` the width is halved until it is (at most
  40 times), else the quantile of a uniform density on ``[mu_1, b_sup]`` is
  used.  ``mu_1`` is the smallest Ritz value
  over the density runs.  The Ritz vectors of the first density run whose
  Ritz value is below ``mu_nev+nex`` replace the leading columns of the start
  block; the remaining columns keep the caller's random vectors.
* The Rayleigh quotient ``G = Q^H A Q`` is Hermitian in exact arithmetic; its
  rounded value is replaced by ``(G + G^H) / 2`` before the eigensolve.
* Random numbers are inputs: the start block ``V`` and the Lanczos start
  vectors are passed in by the caller.

Pins: ``tests/test_oracle_pins.py`` and ``tests/test_oracle_properties.py``
check every function against closed forms, library routines on special
cases, invariants or the paper's worked values.  The width safeguard of the
density-of-states quantile (``dos_estimate``: the halving and the uniform
fallback above) is a reading of a part the paper does not publish; its
arithmetic is pinned by hand-worked cases of each branch
(``tests/golden/dos_safeguard.txt``), while the choice of that heuristic
over the paper's own has nothing in the paper to be checked against.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "shifted_apply",
    "cheb_filter",
    "filter_bounds",
    "degree_one",
    "degrees",
    "householder_qr",
    "jacobi_eigh",
    "rayleigh_ritz",
    "residuals",
    "deflate_and_lock",
    "lanczos_run",
    "dos_cdf",
    "dos_quantile",
    "dos_estimate",
    "lanczos_estimates",
    "solve",
]


# ---------------------------------------------------------------------------
# Chebyshev filter (Sec. 4.1.1, Eq. 7, Alg. 4)
# ---------------------------------------------------------------------------

def shifted_apply(H, X, c):
    """Return ``(H - c I) X`` (the operand of every product in Alg. 4)."""
    return H @ X - c * X


def filter_bounds(b_sup, mu1, mu_nevnex):
    """Alg. 4 lines 2-3: centre ``c``, half-width ``e`` and ``sigma_1``."""
    c = (b_sup + mu_nevnex) / 2.0
    e = (b_sup - mu_nevnex) / 2.0
    sigma1 = e / (mu1 - c)
    return c, e, sigma1


def cheb_filter(H, V, m, b_sup, mu1, mu_nevnex, stats=None):
    """Chebyshev filter with per-column degrees (Alg. 4, recurrence Eq. 7).

    ``V`` is N x b, ``m`` the b column degrees, sorted ascending, each even
    and at least 2 (Alg. 5 line 6 makes them even so that every column ends
    in the buffer that is returned).  Columns ``0 .. s-1`` have reached their
    degree and are left out of later products (Alg. 4 lines 12-14).
    Returns the filtered block (the array Alg. 4 calls W-hat).  If ``stats``
    is a dict, ``stats["matvecs"]`` receives the number of column products
    with ``A`` (the paper's matvec count, Sec. 6.1 footnote 6).
    """
    m = [int(x) for x in m]
    b = V.shape[1]
    if b == 0:
        return V.copy()
    if any(m[i] > m[i + 1] for i in range(b - 1)):
        raise ValueError("degrees must be sorted ascending")
    if any(x < 2 or x % 2 for x in m):
        raise ValueError("degrees must be even and >= 2")
    c, e, sigma1 = filter_bounds(b_sup, mu1, mu_nevnex)
    Vb = np.array(V, dtype=np.complex128, copy=True)
    Wb = (sigma1 / e) * shifted_apply(H, Vb, c)              # line 4
    matvecs = b
    sigma = sigma1                                           # line 5
    s = 0                                                    # line 6
    for i in range(2, m[-1] + 1):                            # line 7
        tau = 1.0 / (2.0 / sigma1 - sigma)                   # line 8
        Vb[:, s:] = (2.0 * tau / e) * shifted_apply(H, Wb[:, s:], c) \
            - (tau * sigma) * Vb[:, s:]                      # line 9
        matvecs += b - s
        Vb, Wb = Wb, Vb                                      # line 10
        sigma = tau                                          # line 11
        while s < b and m[s] <= i:                           # lines 12-14
            s += 1
    if stats is not None:
        stats["matvecs"] = matvecs
    return Wb


# ---------------------------------------------------------------------------
# Degree optimisation (Sec. 4.1.2-4.1.3, Eq. 8, Alg. 5)
# ---------------------------------------------------------------------------

def degree_one(tol, res, lam, c, e, deg_extra=2, deg_max=36):
    """Alg. 5 for one Ritz pair: the smallest even degree meeting Eq. 8."""
    t = (lam - c) / e                                        # line 2
    root = np.sqrt(complex(t * t - 1.0))
    rho = max(abs(t - root), abs(t + root))                  # line 3
    with np.errstate(divide="ignore", invalid="ignore"):
        q = abs(math.log(res / tol) / math.log(rho)) if (rho > 1.0 + 1e-14 and res > 0) \
            else math.inf
    if not math.isfinite(q):
        deg = deg_max
    else:
        deg = int(math.ceil(q))                              # line 4
    deg = min(deg + deg_extra, deg_max)                      # line 5
    deg = deg + deg % 2                                      # line 6
    if deg > deg_max:
        deg -= 2
    return deg


def degrees(resid, ritz, c, e, tol, deg_extra=2, deg_max=36):
    """Alg. 5 applied to every column (Alg. 1 lines 12-14)."""
    return np.array([degree_one(tol, float(r), float(l), c, e, deg_extra, deg_max)
                     for r, l in zip(resid, ritz)], dtype=np.int64)


# ---------------------------------------------------------------------------
# Orthogonalisation: Householder QR (Sec. 3.2, Alg. 1 line 5)
# ---------------------------------------------------------------------------

def householder_qr(X):
    """Thin QR of ``X`` (N x b, N >= b) by complex Householder reflectors.

    Column ``j`` is reduced by ``P_j = I - 2 v v^H`` with
    ``v ~ x - alpha e_1`` and ``alpha = -exp(i arg x_1) ||x||``.  ``Q`` is
    formed by applying the reflectors to the first ``b`` columns of the
    identity in reverse order.  Returns ``(Q, R)``.
    """
    A = np.array(X, dtype=np.complex128, copy=True)
    n, b = A.shape
    if b > n:
        raise ValueError("householder_qr needs N >= b")
    vs = []
    for j in range(b):
        x = A[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -phase * nx
        v = x.copy()
        v[0] -= alpha
        v /= np.linalg.norm(v)
        A[j:, j:] -= 2.0 * np.outer(v, v.conj() @ A[j:, j:])
        vs.append(v)
    R = np.triu(A[:b, :])
    Q = np.zeros((n, b), dtype=np.complex128)
    Q[np.arange(b), np.arange(b)] = 1.0
    for j in reversed(range(b)):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v.conj() @ Q[j:, :])
    return Q, R


# ---------------------------------------------------------------------------
# Small Hermitian eigensolver for Alg. 2 line 3 and the T_k of Alg. 6:
# cyclic complex Jacobi.
# ---------------------------------------------------------------------------

def jacobi_eigh(G, rtol=1e-15, max_sweeps=60):
    """Eigen-decomposition of a Hermitian matrix by cyclic Jacobi rotations.

    Each rotation first removes the phase of ``g_pq`` with
    ``D = diag(1, exp(-i phi))`` and then applies the real symmetric 2 x 2
    rotation that zeroes the (now real) off-diagonal entry.  Sweeps stop when
    ``off(G) <= rtol * ||G||_F``.  Returns ``(w, Z)``, ``w`` ascending and
    ``G = Z diag(w) Z^H``.
    """
    A = np.array(G, dtype=np.complex128, copy=True)
    n = A.shape[0]
    Z = np.eye(n, dtype=np.complex128)
    fro = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = math.sqrt(float(np.sum(np.abs(A - np.diag(np.diag(A))) ** 2)))
        if off <= rtol * fro or n < 2:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                bpq = A[p, q]
                mag = abs(bpq)
                if mag == 0.0:
                    continue
                phase = bpq / mag
                a = A[p, p].real
                d = A[q, q].real
                tau = (d - a) / (2.0 * mag)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # U = diag(1, conj(phase)) @ [[c, s], [-s, c]]
                cp = A[:, p].copy()
                cq = A[:, q].copy()
                A[:, p] = c * cp - s * np.conj(phase) * cq
                A[:, q] = s * cp + c * np.conj(phase) * cq
                rp = A[p, :].copy()
                rq = A[q, :].copy()
                A[p, :] = c * rp - s * phase * rq
                A[q, :] = s * rp + c * phase * rq
                A[p, q] = 0.0
                A[q, p] = 0.0
                A[p, p] = A[p, p].real
                A[q, q] = A[q, q].real
                zp = Z[:, p].copy()
                zq = Z[:, q].copy()
                Z[:, p] = c * zp - s * np.conj(phase) * zq
                Z[:, q] = s * zp + c * np.conj(phase) * zq
    w = np.real(np.diag(A)).copy()
    order = np.argsort(w, kind="stable")
    return w[order], Z[:, order]


# ---------------------------------------------------------------------------
# Rayleigh-Ritz (Alg. 2), residuals (Alg. 1 line 8), locking (Alg. 3)
# ---------------------------------------------------------------------------

def rayleigh_ritz(H, Q):
    """Alg. 2: ``G = Q^H A Q``, ``(W, Lambda) = TSOLVE(G)``, return ``(Q W, Lambda)``."""
    G = Q.conj().T @ (H @ Q)
    G = (G + G.conj().T) / 2.0
    w, Z = jacobi_eigh(G)
    return Q @ Z, w


def residuals(H, V, lam):
    """``Res_a = || A v_a - lambda_a v_a ||_2`` for every column (Alg. 1 line 8)."""
    return np.linalg.norm(H @ V - V * np.asarray(lam)[None, :], axis=0)


def deflate_and_lock(ritz, resid, tol):
    """Alg. 3: stable order by Ritz value, then count the leading pairs with
    ``Res <= tol`` (line 4 returns at the first pair above ``tol``).

    Returns ``(order, n_new)``: the permutation to apply to the active block
    and the number of its leading columns that are locked.
    """
    order = np.argsort(np.asarray(ritz), kind="stable")
    n_new = 0
    for a in order:
        if resid[a] > tol:
            break
        n_new += 1
    return order, n_new


# ---------------------------------------------------------------------------
# Lanczos bounds and density of states (Sec. 4.2, Alg. 6, Eq. 9-10)
# ---------------------------------------------------------------------------

def lanczos_run(H, v0, k):
    """``k`` steps of the Lanczos process ``A U = U T_k + f_k e_k^T``.

    Returns ``(theta, Z, f_norm, U)``: the Ritz values of ``T_k`` (ascending),
    its normalised eigenvectors, ``||f_k||_2`` and the Lanczos basis.
    """
    n = H.shape[0]
    U = np.zeros((n, k), dtype=np.complex128)
    alpha = np.zeros(k)
    beta = np.zeros(k)
    v = np.asarray(v0, dtype=np.complex128) / np.linalg.norm(v0)
    v_prev = np.zeros(n, dtype=np.complex128)
    b_prev = 0.0
    steps = k
    for j in range(k):
        U[:, j] = v
        w = H @ v - b_prev * v_prev
        alpha[j] = np.vdot(v, w).real
        w = w - alpha[j] * v
        beta[j] = np.linalg.norm(w)
        scale = max(np.abs(alpha[:j + 1]).max(), beta[:j + 1].max())
        if beta[j] <= 1e-13 * scale:
            # invariant subspace reached (beta_j is rounding noise): stop here
            steps = j + 1
            break
        v_prev, v = v, w / beta[j]
        b_prev = beta[j]
    T = np.diag(alpha[:steps]) + np.diag(beta[:steps - 1], 1) + np.diag(beta[:steps - 1], -1)
    theta, Z = jacobi_eigh(T.astype(np.complex128))
    return theta, Z, float(beta[steps - 1]), U[:, :steps]


def _normal_cdf(x):
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


def dos_cdf(nodes, t, sig):
    """Integral up to ``t`` of the density estimate of Eq. 10: the average over
    the runs of sum_i w_i Phi((t - theta_i) / sig), with ``nodes`` a list of
    (theta, w) pairs, w_i = |Z_1i|^2."""
    total = 0.0
    for theta, w in nodes:
        total += sum(float(wi) * _normal_cdf((t - float(th)) / sig) for wi, th in zip(w, theta))
    return total / len(nodes)


def dos_quantile(nodes, target, sig):
    """The ``t`` with ``dos_cdf(t) = target`` (Alg. 6 line 11), by bisection."""
    lo = min(float(np.min(th)) for th, _ in nodes) - 10.0 * sig
    hi = max(float(np.max(th)) for th, _ in nodes) + 10.0 * sig
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if dos_cdf(nodes, mid, sig) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def dos_estimate(nodes, target, mu1, b_sup, sigma=0.25):
    """``mu_nev+nex`` of Alg. 6 line 11: the ``target`` quantile of the
    density estimate of Eq. 10 built from ``nodes`` (one (theta, w) pair of
    arrays per density run), kept strictly inside ``(mu_1, b_sup)``.

    The Gaussian width is ``sigma`` times the half-width of ``[mu_1,
    b_sup]`` (``sigma`` itself when that interval has collapsed).  Sec. 4.2
    leaves the safeguards unpublished.  Reading: when the quantile is not
    inside the interval by a margin of ``1e-6 (b_sup - mu_1)``, halve the
    width and take the quantile again, at most 40 times; failing that, take
    the ``target`` quantile of a uniform density on ``[mu_1, b_sup]``, with
    ``target`` clamped to ``[1e-3, 0.5]``.

    Returns ``{"mu": value, "halvings": count, "fallback": bool}``.
    """
    half = (b_sup - mu1) / 2.0
    # a collapsed interval (all Ritz values equal) falls back to sigma itself
    sig = sigma * half if half > 1e-12 * max(1.0, abs(b_sup), abs(mu1)) else sigma
    mu = dos_quantile(nodes, target, sig)
    margin = 1e-6 * (b_sup - mu1)
    halvings = 0
    while not (mu1 + margin < mu < b_sup - margin) and halvings < 40:
        sig *= 0.5
        halvings += 1
        mu = dos_quantile(nodes, target, sig)
    if mu1 + margin < mu < b_sup - margin:
        return {"mu": mu, "halvings": halvings, "fallback": False}
    return {"mu": mu1 + (b_sup - mu1) * min(max(target, 1e-3), 0.5), "halvings": halvings,
            "fallback": True}


def lanczos_estimates(H, starts, k, nvec, approx, nev, nex, V=None, sigma=0.25):
    """Alg. 6: spectral bounds, and (when ``approx`` is false) the density
    estimate of Eq. 10 with ``mu_1``, ``mu_nev+nex`` and start vectors.

    ``starts`` holds ``1 + nvec`` start vectors as columns (column 0 for the
    bound run of line 2, columns ``1..nvec`` for the runs of line 8).
    Returns a dict with ``b_sup``, ``mu1``, ``mu_nevnex`` (None when
    ``approx``), ``V`` (the start block with Ritz vectors interspersed) and
    ``theta_absmax`` (largest |theta| seen).
    """
    n = H.shape[0]
    theta0, _, f0, _ = lanczos_run(H, starts[:, 0], k)
    b_sup = f0 + float(theta0.max())                         # line 3
    absmax = float(np.abs(theta0).max())
    out = {"b_sup": b_sup, "mu1": None, "mu_nevnex": None, "V": V,
           "theta_absmax": absmax, "matvecs": k}
    if approx:                                               # lines 4-6
        return out
    runs = [lanczos_run(H, starts[:, 1 + j], k) for j in range(nvec)]   # lines 7-9
    out["matvecs"] = k * (1 + nvec)
    for theta, _, f, _ in runs:
        b_sup = max(b_sup, f + float(theta.max()))
        absmax = max(absmax, float(np.abs(theta).max()))
    mu1 = min(float(theta.min()) for theta, _, _, _ in runs)             # line 12
    target = (nev + nex) / n                                 # line 11
    nodes = [(theta, np.abs(Z[0, :]) ** 2) for theta, Z, _, _ in runs]
    mu_nevnex = dos_estimate(nodes, target, mu1, b_sup, sigma)["mu"]
    Vout = None
    if V is not None:                                        # line 13
        Vout = np.array(V, dtype=np.complex128, copy=True)
        theta1, Z1, _, U1 = runs[0]
        sel = [i for i in range(len(theta1)) if theta1[i] < mu_nevnex][: Vout.shape[1]]
        for col, i in enumerate(sel):
            Vout[:, col] = U1 @ Z1[:, i]
    out.update(b_sup=b_sup, mu1=mu1, mu_nevnex=mu_nevnex, V=Vout, theta_absmax=absmax)
    return out


# ---------------------------------------------------------------------------
# The ChASE driver (Alg. 1)
# ---------------------------------------------------------------------------

def solve(H, nev, nex, V, lanczos_starts, tol=1e-10, Lam=None, approx=False,
          deg=20, optim=True, deg_extra=2, deg_max=36, max_iter=25,
          lanczos_iter=25, num_lanczos=4, dos_sigma=0.25, conv_mode="rel"):
    """Alg. 1 with the locked-prefix layout of Sec. 5.1.1.

    ``V`` (N x (nev+nex)) is the start block: random vectors when ``approx``
    is false, the previous problem's vectors otherwise (``Lam`` then holds the
    previous Ritz values, whose min and max give ``mu_1``, ``mu_nev+nex``,
    Sec. 3.3).  Returns a dict with the Ritz values (ascending), Ritz vectors,
    residuals, the number of locked pairs, iterations and matvecs.
    """
    H = np.asarray(H, dtype=np.complex128)
    n = H.shape[0]
    nx = nev + nex
    V = np.array(V, dtype=np.complex128, copy=True)
    d0 = int(deg) + int(deg) % 2
    m = np.full(nx, d0, dtype=np.int64)                      # line 1
    est = lanczos_estimates(H, lanczos_starts, lanczos_iter, num_lanczos,
                            approx, nev, nex, V=None if approx else V,
                            sigma=dos_sigma)                 # line 2
    b_sup = est["b_sup"]
    h = est["theta_absmax"]
    matvecs = est["matvecs"]
    if approx:
        lam_in = np.asarray(Lam, dtype=np.float64)
        mu1, mu_nn = float(lam_in.min()), float(lam_in.max())
    else:
        mu1, mu_nn, V = est["mu1"], est["mu_nevnex"], est["V"]
    ritz = np.zeros(nx)
    res = np.full(nx, np.inf)
    nconv = 0
    it = 0
    filter_matvecs = 0
    while nconv < nev and it < max_iter:                     # line 3
        it += 1
        act = slice(nconv, nx)
        degs = m[nconv:]
        V[:, act] = cheb_filter(H, V[:, act], degs, b_sup, mu1, mu_nn)    # line 4
        fm = int(degs.sum())
        filter_matvecs += fm
        Q, _ = householder_qr(V)                             # line 5
        Qt = Q[:, nconv:]                                    # line 6
        Vn, lt = rayleigh_ritz(H, Qt)                        # line 7
        rt = residuals(H, Vn, lt)                            # line 8
        matvecs += fm + 2 * (nx - nconv)
        h = max(h, float(np.abs(lt).max()))
        tol_eff = tol * h if conv_mode == "rel" else tol
        order, n_new = deflate_and_lock(lt, rt, tol_eff)     # line 9 (Alg. 3)
        V[:, act] = Vn[:, order]
        ritz[act] = lt[order]
        res[act] = rt[order]
        nconv += n_new
        mu1 = float(ritz.min())                              # line 10
        mu_nn = float(ritz.max())
        c = (b_sup + mu_nn) / 2.0                            # line 11
        e = (b_sup - mu_nn) / 2.0
        if nconv < nx:
            if optim:                                        # lines 12-14
                m[nconv:] = degrees(res[nconv:], ritz[nconv:], c, e, tol_eff,
                                    deg_extra, deg_max)
            else:
                m[nconv:] = d0
            order2 = np.argsort(m[nconv:], kind="stable")    # line 15
            idx = nconv + order2
            V[:, nconv:] = V[:, idx]
            ritz[nconv:] = ritz[idx]
            res[nconv:] = res[idx]
            m[nconv:] = m[idx]
    final = np.argsort(ritz, kind="stable")
    return {
        "ritz": ritz[final],
        "V": V[:, final],
        "resid": res[final],
        "nconv": nconv,
        "iterations": it,
        "matvecs": matvecs,
        "filter_matvecs": filter_matvecs,
        "b_sup": b_sup,
        "converged": nconv >= nev,
        "tol_eff": tol * h if conv_mode == "rel" else tol,
    }
