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
"""
import numpy as np

REL = 1e-4
LL_ABS = 1e-5


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
