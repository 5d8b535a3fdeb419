"""Comparison helpers for GPU-vs-oracle parity (shared by the GPU tests).

Tolerances (per component b, GPU binary32 with binary64 finalize vs the FP64
oracle, from identical initial parameters):
  |d pi_b|        <= rel * pi_b + 1e-7
  ||d mu_b||_2    <= rel * ||mu_b||_2 + 1e-6 m
  ||d Sigma_b||_F <= rel * ||Sigma_b||_F
  |d l|           <= 1e-5   (mean per-point log-likelihood, absolute)
with rel = 1e-4.  Components with pi_b < live_floor are numerically
undetermined in binary32 (their responsibilities sit below binary32
resolution); they are compared only for validity (finite, symmetric, PD).

Per-point log-likelihoods are compared against ``per_point_bound``, a bound on
the rounding error of the E-step's binary32 arithmetic at each point (below).
"""
import numpy as np

REL = 1e-4
LL_ABS = 1e-5

U32 = 2.0 ** -24          # unit roundoff of binary32
EPS_EX2 = 2.0 ** -21      # relative error allowed for ex2.approx (the hardware's is about 2^-22)
EPS_LG2 = 2.0 ** -21      # absolute error allowed for lg2.approx near 1 (about 2^-22 in hardware)
ALPHA = np.sqrt(np.log2(np.e) / 2.0)


def per_point_bound(pts, weights, means, covs, form="d", chunk_pairs=1 << 21):
    """Bound on |l_n(GPU) - l_n(exact)| for the per-point log-likelihood of each point.

    The E-step (Eq. logestep with the log-density of Eq. simplifiedGaussian) works in
    base 2 with binary32 operands: P' = alpha L^-1 and b' = -P' mu are formed in
    binary64 and rounded to binary32 (alpha = sqrt(log2(e) / 2)); y = P' x + b'
    ("b" form, 3-D fit and log-likelihood path) or y = P' (x - mu) ("d" form, 4-D
    path) by a chain of at most D fused multiply-adds; q' = |y|^2 + (c_max - c_b) by D
    more; e = ex2(-q'); the sum over components by a tree of additions; l = ln 2 *
    (lg2(sum) + reference).  Rounding error terms, u = 2^-24:
      |dy_i|  <= 5u S_i,  S_i = sum_j |P'_ij x_j| + |b'_i|  (b form)  or  sum_j |P'_ij| |x_j - mu_j|  (d form)
                (input rounding of P' and b' or of x - mu: u S_i; the chain: D u S_i)
      |dq'|   <= sum_i (2 |y_i| |dy_i| + dy_i^2) + 3u (|y|^2 + c') + u (|c_b| + c')
      |dl_n|  <= ln2 sum_b gamma_nb |dq'_nb| + eps_ex2 + (log2 K + 12) u      (sum of e, chunk combine)
                 + ln2 (eps_lg2 + u |c_max| + (log2 K + 10) u)                  (lg2, the reference)
                 + 2u |l_n|                                                     (final add, scaling by ln 2)
    gamma (responsibilities), y and c are evaluated here in binary64 from the same
    binary32 inputs the GPU received.  The bound is a first-order worst case (every
    rounding in the same direction); the GPU's actual errors are usually much smaller.
    Returns the bound per point (binary64)."""
    X = np.asarray(pts, np.float64)
    w = np.asarray(weights, np.float64)
    mu = np.asarray(means, np.float64)
    S = np.asarray(covs, np.float64)
    N, D = X.shape
    K = len(w)
    Lc = np.linalg.cholesky(S)
    P = np.linalg.inv(Lc)
    P = np.tril(P)
    Q = ALPHA * P                                     # K x D x D
    bq = -np.einsum("bij,bj->bi", Q, mu)              # b' (K x D)
    logdiag = np.log2(np.diagonal(P, axis1=1, axis2=2)).sum(1)
    c = np.log2(w) + logdiag - 0.5 * D * np.log2(2 * np.pi)
    cmax = c.max()
    cp = cmax - c
    absQ = np.abs(Q)
    lnw_norm = np.log(w) + np.log(np.diagonal(P, axis1=1, axis2=2)).sum(1) - 0.5 * D * np.log(2 * np.pi)
    out = np.empty(N)
    step = max(1, chunk_pairs // K)
    for a in range(0, N, step):
        x = X[a:a + step]
        d = x[:, None, :] - mu[None]                  # n x K x D
        y = np.einsum("bij,nbj->nbi", Q, d)
        if form == "b":
            Si = np.einsum("bij,nj->nbi", absQ, np.abs(x)) + np.abs(bq)[None]
        else:
            Si = np.einsum("bij,nbj->nbi", absQ, np.abs(d))
        dy = 5 * U32 * Si
        q = (y * y).sum(-1)
        dq = (2 * np.abs(y) * dy + dy * dy).sum(-1) + 3 * U32 * (q + cp[None]) + U32 * (np.abs(c) + cp)[None]
        logp = lnw_norm[None] - q / np.log2(np.e)     # ln(pi_b N(x | b)) = lnw_norm - q / log2(e)
        m = logp.max(1, keepdims=True)
        e = np.exp(logp - m)
        tot = e.sum(1, keepdims=True)
        g = e / tot
        l = (m + np.log(tot))[:, 0]
        lk = np.log2(K)
        out[a:a + step] = (np.log(2) * (g * dq).sum(1) + EPS_EX2 + (lk + 12) * U32
                           + np.log(2) * (EPS_LG2 + U32 * abs(cmax) + (lk + 10) * U32) + 2 * U32 * np.abs(l))
    return out


def to_np(x):
    if hasattr(x, "detach"):
        return x.detach().cpu().numpy()
    return np.asarray(x)


def model_mismatches(got, ref, rel=REL, live_floor=1e-6):
    w, m, c = (to_np(a).astype(np.float64) for a in got)
    rw, rm, rc = (np.asarray(a, np.float64) for a in ref)
    K = len(rw)
    bad = []
    for b in range(K):
        if not (np.all(np.isfinite(m[b])) and np.all(np.isfinite(c[b])) and np.isfinite(w[b])):
            bad.append((b, "non-finite"))
            continue
        if rw[b] < live_floor:
            if np.any(np.linalg.eigvalsh(0.5 * (c[b] + c[b].T)) <= 0):
                bad.append((b, "dead component not PD"))
            continue
        dw = abs(w[b] - rw[b])
        dm = np.linalg.norm(m[b] - rm[b])
        dc = np.linalg.norm(c[b] - rc[b])
        if dw > rel * rw[b] + 1e-7:
            bad.append((b, f"weight {w[b]:.9g} vs {rw[b]:.9g} (rel {dw / rw[b]:.2e})"))
        if dm > rel * np.linalg.norm(rm[b]) + 1e-6:
            bad.append((b, f"mean diff {dm:.3e} vs |mu| {np.linalg.norm(rm[b]):.3e}"))
        if dc > rel * np.linalg.norm(rc[b]):
            bad.append((b, f"cov rel diff {dc / np.linalg.norm(rc[b]):.2e}"))
    return bad


def assert_model_close(got, ref, rel=REL, live_floor=1e-6):
    bad = model_mismatches(got, ref, rel, live_floor)
    assert not bad, f"{len(bad)} components outside tolerance: {bad[:12]}"


def max_rel_errors(got, ref):
    w, m, c = (to_np(a).astype(np.float64) for a in got)
    rw, rm, rc = (np.asarray(a, np.float64) for a in ref)
    ew = np.max(np.abs(w - rw) / np.maximum(rw, 1e-30))
    em = np.max(np.linalg.norm(m - rm, axis=1) / np.maximum(np.linalg.norm(rm, axis=1), 1e-30))
    ec = np.max(np.linalg.norm((c - rc).reshape(len(rw), -1), axis=1) / np.linalg.norm(rc.reshape(len(rw), -1), axis=1))
    return ew, em, ec
