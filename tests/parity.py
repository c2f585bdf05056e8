"""Comparison rules of the CUDA path against the FP64 oracle.

Every form computes the covariance C with some error dC; the later stages
only propagate it.  E_COV[form] bounds that error in the spectral norm,
relative to lambda_1 (||C - C*||_2 <= E_COV lambda_1; measured for each form
by tests/test_gpu_stages.py, which asserts it).  The bounds below follow from
it by perturbation theory of the symmetric eigenproblem:

  eigenvalues, i <= k, outside a degenerate cluster: the per-eigenvalue
      relative error |lam_i - lam*_i| / lam*_i <= max(LAM_TOL, E_COV lam*_1 /
      lam*_i).  LAM_TOL is the target (P64 1e-10, MIX 2e-5, P32 2e-3); the
      second term is Weyl's inequality |dlam_i| <= ||dC||_2, which makes a
      small eigenvalue of an FP32-class covariance (MIX, P32) miss the target
      by lam*_1/lam*_i -- stated, not hidden: the metrics report the worst
      ratio to the target and whether every component met it.
  all eigenvalues, relative to lam_1: P64 <= 1e-7, MIX <= 1e-4, P32 <= 2e-3
      (near-degenerate clusters -- the noise floor -- are not resolved by the
      FP64 refinement, whose threshold delta treats them as one subspace)
  means: |mu - mu*| <= MU_TOL * max|mu*|
  eigenvectors: after sign normalisation, individually only where the
      relative gap min(lam_{j-1}-lam_j, lam_j-lam_{j+1})/lam_1 >= 1e3 eps_form,
      with |v - v*|_max <= c * eps_form / gap (first-order perturbation);
      elsewhere the subspace of the cluster is compared.
  projection, component j <= k with an individually pinned vector:
      max_n |Q_nj - Q*_nj| / max_n |Q*_nj| <= max(1e-4, q_bound_j), each
      column against its own scale.  First order, v_j moves by
      sum_i (v_i^T dC v_j)/(lam_j - lam_i) v_i, so column j of Q picks up
      column i scaled by that coefficient; relative to column j's own scale
      (max |Q_j| ~ sqrt(lam_j)) the error is at most
          q_bound_j = 1e-5 + 4 E_COV lam_1 max_{i != j} sqrt(lam_i/lam_j) / |lam_i - lam_j|
      (1e-5: the FP32 arithmetic of the projection kernel; 4: the spread of
      max |Q_i| / sqrt(lam_i) over columns).  Where the target of 1e-4 is
      reachable it is the bound; below, q_bound_j is, and the metrics say so.
"""
import numpy as np

EPS = {"p64": 1e-15, "mix": 1e-7, "p32": 1e-6}
LAM_TOL = {"p64": 1e-10, "mix": 2e-5, "p32": 2e-3}
# ||C - C*||_2 / lam_1 of each covariance form (asserted by the covariance stage
# test).  MIX: FP32 accumulation runs of 8 chunks on FP32 cubes, measured up to
# 1.5e-6 (exact products and sums on 16-bit cubes); P32: FP32 SIMT partials.
E_COV = {"p64": 1e-13, "mix": 5e-6, "p32": 2e-6}
MU_TOL = {"p64": 1e-12, "mix": 1e-6, "p32": 1e-6}
LAM_ALL_TOL = {"p64": 1e-7, "mix": 1e-4, "p32": 2e-3}
ORTH_TOL = {"p64": 1e-11, "mix": 1e-6, "p32": 1e-4}
Q_TOL = 1e-4           # the stated projected-cube bound
Q_ARITH = 1e-5         # FP32 arithmetic of the projection kernel, per column


def lam_bounds(lam_ref, k, form):
    """Per-eigenvalue relative bounds of the first k eigenvalues (see above)."""
    lam_ref = np.asarray(lam_ref, dtype=np.float64)
    l1 = max(abs(lam_ref[0]), 1e-300)
    weyl = E_COV[form] * l1 / np.maximum(np.abs(lam_ref[:k]), 1e-300)
    return np.maximum(LAM_TOL[form], weyl)


def q_bounds(lam_ref, k, form):
    """Per-component bounds of the projection error (see above)."""
    lam = np.maximum(np.asarray(lam_ref, dtype=np.float64), 0.0)
    l1 = max(lam[0], 1e-300)
    out = np.empty(k)
    for j in range(k):
        if lam[j] <= 0.0:
            out[j] = np.inf
            continue
        others = np.delete(np.arange(lam.shape[0]), j)
        gap = np.abs(lam[others] - lam[j])
        with np.errstate(divide="ignore"):
            amp = np.where(gap > 0, np.sqrt(lam[others] / lam[j]) / gap, np.inf)
        out[j] = max(Q_TOL, Q_ARITH + 4.0 * E_COV[form] * l1 * amp.max())
    return out


def rel_gaps(lam):
    lam = np.asarray(lam, dtype=np.float64)
    l1 = max(abs(lam[0]), 1e-300)
    d = np.abs(np.diff(lam)) / l1
    left = np.concatenate([[np.inf], d])
    right = np.concatenate([d, [np.inf]])
    return np.minimum(left, right)


def sign_norm(V):
    V = np.array(V, dtype=np.float64, copy=True)
    idx = np.argmax(np.abs(V), axis=0)
    sg = np.sign(V[idx, np.arange(V.shape[1])])
    sg[sg == 0] = 1
    return V * sg[None, :]


def subspace_dist(V1, V2):
    P1 = V1 @ V1.T
    P2 = V2 @ V2.T
    return np.linalg.norm(P1 - P2, 2)


def compare(gpu, ref, k, form, check_q=True, lam_floor=None, orth_tol=None, vec_eps=None):
    """gpu = (mu, lam, V, Q) numpy float64; ref = oracle.pca_fit dict.  Returns metrics,
    raises AssertionError on a violation.  lam_floor (a fraction of lam_1): eigenvalues
    below it are measured against lam_floor * lam_1 instead of themselves;
    orth_tol replaces ORTH_TOL[form] and vec_eps the eps of the eigenvector bound."""
    mu, lam, V, Q = gpu
    m = {}
    lam_ref = ref["lam"]
    B = lam_ref.shape[0]
    mu_scale = max(np.abs(ref["mu"]).max(), 1e-30)
    m["mu_err"] = float(np.abs(mu - ref["mu"]).max() / mu_scale)
    assert m["mu_err"] <= MU_TOL[form], m

    gaps = rel_gaps(lam_ref)
    eps = EPS[form]
    pinned = gaps >= 1e3 * eps
    kk = min(k, B)
    l1 = max(abs(lam_ref[0]), 1e-300)
    # eigenvalue error: per eigenvalue for i <= k outside clusters (target, or
    # Weyl's bound where the form's covariance error does not allow the target),
    # relative to lam_1 for all
    floor = lam_floor * l1 if lam_floor else 0.0
    rel = np.abs(lam[:kk] - lam_ref[:kk]) / np.maximum(np.maximum(np.abs(lam_ref[:kk]), floor),
                                                         1e-300)
    bnd = lam_bounds(lam_ref, kk, form)
    sel = pinned[:kk]
    m["lam_rel_topk"] = float(rel[sel].max()) if sel.any() else 0.0
    m["lam_rel_topk_over_target"] = float((rel[sel] / LAM_TOL[form]).max()) if sel.any() else 0.0
    m["lam_target_met"] = bool(m["lam_rel_topk_over_target"] <= 1.0)
    m["lam_rel_l1_all"] = float(np.abs(lam - lam_ref).max() / l1)
    if l1 > 0:
        assert np.all(rel[sel] <= bnd[sel]), (m, rel, bnd)
        assert m["lam_rel_l1_all"] <= LAM_ALL_TOL[form], m
    else:
        assert np.all(lam == 0.0)
    # orthogonality of the returned eigenvectors
    m["orth"] = float(np.abs(V.T @ V - np.eye(B)).max())
    assert m["orth"] <= (orth_tol if orth_tol is not None else ORTH_TOL[form]), m
    # eigenvectors: individually where separated, else subspace of the top-k
    Vs, Vr = sign_norm(V), ref["V"]
    vec_err = 0.0
    for j in range(kk):
        if pinned[j]:
            ve = vec_eps if vec_eps is not None else eps
            bound = max(200.0 * ve / gaps[j], 20.0 * ve)
            err = float(np.abs(Vs[:, j] - Vr[:, j]).max())
            vec_err = max(vec_err, err / bound)
    m["vec_err_over_bound"] = vec_err
    assert vec_err <= 1.0, m
    m["subspace_k"] = float(subspace_dist(V[:, :kk], Vr[:, :kk]))
    if check_q and Q is not None:
        qb = q_bounds(lam_ref, kk, form)
        qerr, qover = 0.0, 0.0
        for j in range(kk):
            if not pinned[j]:
                continue
            # both sides sign-normalised: flip Q column when the vector was flipped
            sgn = 1.0 if np.dot(V[:, j], Vr[:, j]) >= 0 else -1.0
            scale = max(np.abs(ref["Q"][:, j]).max(), 1e-30)
            e = float(np.abs(sgn * Q[:, j] - ref["Q"][:, j]).max() / scale)
            qerr = max(qerr, e)
            qover = max(qover, e / Q_TOL)
            assert e <= qb[j], (m, j, e, qb[j])
        m["q_err"] = qerr
        m["q_err_over_target"] = qover
    return m
