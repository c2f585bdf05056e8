"""Comparison rules of the CUDA path against the FP64 oracle.

Tolerances (per precision form):
  eigenvalues, i <= k, outside a degenerate cluster: relative error
      P64 <= 1e-10, MIX <= 2e-5 of lam_1 (the two-term BF16 split of the
      covariance carries ~2^-17 relative error per element, so the bound is
      absolute: relative for the leading component, proportionally looser
      below it), P32 <= 2e-3 (plain FP32, no refinement)
  all eigenvalues, relative to lam_1: P64 <= 1e-7, MIX <= 1e-4, P32 <= 2e-3
      (near-degenerate clusters -- the noise floor -- are not resolved by the
      FP64 refinement, whose threshold delta treats them as one subspace)
  means: |mu - mu*| <= tol_mu * max|mu*|
  eigenvectors: after sign normalisation, individually only where the
      relative gap min(lam_{j-1}-lam_j, lam_j-lam_{j+1})/lam_1 >= 1e3 eps_form,
      with |v - v*|_max <= c * eps_form / gap (first-order perturbation);
      elsewhere the subspace of the cluster is compared.
  projection, component j <= k with an individually pinned vector:
      max_n |Q_nj - Q*_nj| / max_n |Q*_nj| <= 1e-4 (P64), 1e-2 (P32);
      MIX: max_n |Q_nj - Q*_nj| / max_n |Q*_n1| <= 1e-4 (normalised by the
      leading component, like its eigenvalues)
"""
import numpy as np

EPS = {"p64": 1e-15, "mix": 1e-7, "p32": 1e-6}
LAM_TOL = {"p64": 1e-10, "mix": 2e-5, "p32": 2e-3}
MU_TOL = {"p64": 1e-12, "mix": 1e-6, "p32": 1e-6}
LAM_ALL_TOL = {"p64": 1e-7, "mix": 1e-4, "p32": 2e-3}
ORTH_TOL = {"p64": 1e-11, "mix": 1e-6, "p32": 1e-4}
Q_TOL = {"p64": 1e-4, "mix": 1e-4, "p32": 1e-2}


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
    below it are held to LAM_TOL * lam_floor * lam_1 absolute instead of relative;
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
    # eigenvalue error: relative for i <= k outside clusters, relative to lam_1 for all
    # MIX: the two-term BF16 split bounds the covariance at ~2^-17 per element,
    # so its eigenvalue errors are ~2e-5 of lam_1 in absolute terms
    floor = l1 if form == "mix" else (lam_floor * l1 if lam_floor else 0.0)
    rel = np.abs(lam[:kk] - lam_ref[:kk]) / np.maximum(np.maximum(np.abs(lam_ref[:kk]), floor),
                                                         1e-300)
    m["lam_rel_topk"] = float(rel[pinned[:kk]].max()) if pinned[:kk].any() else 0.0
    m["lam_rel_l1_all"] = float(np.abs(lam - lam_ref).max() / l1)
    if l1 > 0:
        assert m["lam_rel_topk"] <= LAM_TOL[form], m
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
        qerr = 0.0
        for j in range(kk):
            if not pinned[j]:
                continue
            # both sides sign-normalised: flip Q column when the vector was flipped
            sgn = 1.0 if np.dot(V[:, j], Vr[:, j]) >= 0 else -1.0
            # MIX: errors scale with the leading component (see the eigenvalue note)
            scale = max(np.abs(ref["Q"][:, 0 if form == "mix" else j]).max(), 1e-30)
            qerr = max(qerr, float(np.abs(sgn * Q[:, j] - ref["Q"][:, j]).max() / scale))
        m["q_err"] = qerr
        assert qerr <= Q_TOL[form], m
    return m
