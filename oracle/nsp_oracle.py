"""FP64 CPU oracle of the two-level Nyström–Schur preconditioner (Al Daas, Rees & Scott).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
It shares no code with the CUDA path (it does not import the package
``paper_2101_12164_gb300``) and the product path never calls it.

Everything here is plain, slow and follows the paper step by step in float64:

* ``DBBD``                 : the block form of §2.3, eq. (perm_A), and the Schur
                             complements S_Gamma (§2.3, eq. (schur_complement)) and S_I (§4.1, eq. (SI)).
* ``block_pcg``            : breakdown-free block PCG (cited in §5.1 as Ji & Li 2017,
                             O'Leary 1980; the paper prints no listing, our reading is in
                             the docstring).
* ``nystrom_core``         : Algorithm 2 steps 5-10 (= Algorithm 1 steps 3-8).
* ``build_m2``             : Algorithm 2, in the paper's S_I form (step 3) or the
                             equivalent S_Gamma correction form (SMW identity, §4.1 eq. (S-1)),
                             optionally with q power iterations (§2.1 eq. (power)).
* ``build_m1``             : the variant M1 of §4.1 with a dense R_Gamma (small interfaces).
* ``build_m3``             : the variant M3 of §4.3 (Nyström on S_I^{-1}), and M_{3A-DEF}.
* ``recursive_gamma``      : the recursive treatment of A_Gamma (concluding section): A_Gamma^{-1}
                             replaced by a block elimination of A_Gamma's own DBBD split whose
                             Schur solve is that split's M2 (``NestedGammaInverse``).
* ``M2ADEF``               : the adapted-deflation variant M_{2A-DEF} of §4.3 (defined
                             like eq. (deflation_comp_from_low_rank) and eq.
                             (our_two_level_preconditioner), moved through Z = A_G^{-1} U).
* ``pcg``                  : outer PCG on S_Gamma w = f (§2.3 eq. (Sx=b)) with M2 (§4.3 eq. (left_prec_mat)).
* ``solve``                : block elimination of §2.3 eq. (A_LDLT) around the outer PCG.
* ``solve_full_space``     : PCG on A with the block-factorization preconditioner of §2.3
                             whose Schur block is M2 (a reading used by the GPU's
                             mixed-precision outer solve; equal iterates in exact arithmetic).
* ``lanczos_tridiagonal``,
  ``kappa_estimate``       : the condition number of the preconditioned operator (the
                             kappa of the CG error bound eq. (k-th_error_cg) of §1, and the
                             kappa_eff of §4.2) estimated from the outer PCG's coefficients,
                             whose Lanczos tridiagonal has the extreme Ritz values.

Library primitives used as single steps: SuperLU sparse direct solves (for A_I^{-1},
A_Gamma^{-1}), numpy QR, symmetric EVD, dense Cholesky, matrix products.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ----------------------------------------------------------------------------------------
# §2.3, eq. (perm_A): doubly bordered block diagonal form
# ----------------------------------------------------------------------------------------
class NotDBBD(ValueError):
    pass


def _lu(M):
    """Sparse direct factorization of an SPD block (SuperLU, symmetric mode)."""
    M = sp.csc_matrix(M)
    if M.shape[0] == 0:
        return None
    return spla.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                     options=dict(SymmetricMode=True))


class DBBD:
    """Split A by ``part`` into A_I (block diagonal), A_IG, A_GI, A_G (§2.3, eq. (perm_A)).

    Interior unknowns are ordered block by block, each block in increasing original
    index; interface unknowns (part < 0) in increasing original index.
    """

    def __init__(self, A, part, nblocks=None):
        A = sp.csr_matrix(A, dtype=np.float64)
        part = np.asarray(part)
        self.n = A.shape[0]
        self.nblocks = int(part.max()) + 1 if nblocks is None else int(nblocks)
        self.gamma = np.nonzero(part < 0)[0]
        self.blocks = [np.nonzero(part == b)[0] for b in range(self.nblocks)]
        self.interior = np.concatenate(self.blocks) if self.blocks else np.zeros(0, int)
        self.offsets = np.cumsum([0] + [len(b) for b in self.blocks])
        I, G = self.interior, self.gamma
        self.A = A
        self.A_I = A[I][:, I].tocsr()
        self.A_IG = A[I][:, G].tocsr()
        self.A_GI = A[G][:, I].tocsr()
        self.A_G = A[G][:, G].tocsr()
        self.n_I, self.n_G = len(I), len(G)
        # A_I must be block diagonal: no coupling between different subdomains.
        blk = np.repeat(np.arange(self.nblocks), np.diff(self.offsets))
        coo = self.A_I.tocoo()
        if np.any(blk[coo.row] != blk[coo.col]):
            raise NotDBBD("interior blocks are coupled: partition is not DBBD")
        self._blk_lu = [_lu(self.A_I[o:e][:, o:e]) for o, e in
                        zip(self.offsets[:-1], self.offsets[1:])]
        self._g_lu = _lu(self.A_G)

    # A_I^{-1} B, block by block ("factorized cheaply in parallel", §2.3)
    def solve_I(self, B):
        B = np.asarray(B, dtype=np.float64)
        X = np.empty_like(B)
        for lu, o, e in zip(self._blk_lu, self.offsets[:-1], self.offsets[1:]):
            if e > o:
                X[o:e] = lu.solve(np.ascontiguousarray(B[o:e]))
        return X

    # A_Gamma^{-1} B: the first-level preconditioner S1^{-1} of §2.3 eq. (S1)
    def solve_G(self, B):
        return self._g_lu.solve(np.ascontiguousarray(np.asarray(B, dtype=np.float64)))

    # S_Gamma = A_G - A_GI A_I^{-1} A_IG (§2.3, eq. (schur_complement)), applied to a block
    def apply_S_gamma(self, X):
        return self.A_G @ X - self.A_GI @ self.solve_I(self.A_IG @ X)

    # S_I = A_I - A_IG A_G^{-1} A_GI (§4.1, eq. (SI)), applied to a block
    def apply_S_I(self, X):
        return self.A_I @ X - self.A_IG @ self.solve_G(self.A_GI @ X)

    # dense forms for tiny problems
    def dense_S_gamma(self):
        return self.A_G.toarray() - self.A_GI.toarray() @ self.solve_I(self.A_IG.toarray())

    def dense_S_I(self):
        return self.A_I.toarray() - self.A_IG.toarray() @ self.solve_G(self.A_GI.toarray())


def block_cholesky(A_block, order):
    """Dense lower Cholesky factor of A_block[order][:, order] (numpy; tiny/sampled use)."""
    M = sp.csr_matrix(A_block)[order][:, order].toarray()
    return np.linalg.cholesky(M)


# ----------------------------------------------------------------------------------------
# Breakdown-free block PCG (§5.1: "breakdown-free block PCG", refs. Ji & Li 2017, O'Leary
# 1980). Reading (the paper prints no listing):
#   R0 = B - A X0, Z0 = M R0, P0 = orth(Z0)
#   loop:  Q = A P;  alpha = (P^T Q)^{-1} P^T R;  X += P alpha;  R -= Q alpha
#          stop when max_j ||R_j|| / ||B_j|| <= tol
#          Z = M R;  beta = -(P^T Q)^{-1} Q^T Z;  P = orth(Z + P beta)
# orth(W): Cholesky-QR of W^T W taken column by column; a column whose pivot is
# <= drop_tol * (its squared norm) lies (numerically) in the span of the kept columns and
# is dropped, so P loses columns instead of breaking down.
# ----------------------------------------------------------------------------------------
def kept_columns(C, drop_tol=1e-12):
    """Columns j of the Gram matrix C whose pivot, after eliminating the columns kept before
    j, exceeds drop_tol * C[j, j] (the rule of the thresholded Cholesky-QR below)."""
    s = C.shape[0]
    keep = []
    for j in range(s):
        if C[j, j] <= 0.0:
            continue
        # pivot of column j after eliminating the kept ones (Schur complement)
        if keep:
            Ck = C[np.ix_(keep, keep)]
            c = C[keep, j]
            piv = C[j, j] - c @ np.linalg.solve(Ck, c)
        else:
            piv = C[j, j]
        if piv > drop_tol * C[j, j]:
            keep.append(j)
    return keep


def orth(W, drop_tol=1e-12):
    """Orthonormal basis of the columns of W kept by a thresholded Cholesky-QR."""
    C = W.T @ W
    keep = kept_columns(C, drop_tol)
    if not keep:
        return W[:, :0]
    R = np.linalg.cholesky(C[np.ix_(keep, keep)]).T       # upper: C_kk = R^T R
    return sla.solve_triangular(R, W[:, keep].T, trans="T", lower=False).T


def block_pcg(apply_A, apply_M, B, tol, maxit=500, drop_tol=1e-12, X0=None):
    """Returns (X, iterations, history of max relative column residuals)."""
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64)
    R = B - apply_A(X) if X0 is not None else B.copy()
    bn = np.linalg.norm(B, axis=0)
    bn[bn == 0] = 1.0
    hist = [float(np.max(np.linalg.norm(R, axis=0) / bn))]
    if hist[-1] <= tol:
        return X, 0, hist
    P = orth(apply_M(R), drop_tol)
    it = 0
    while it < maxit and P.shape[1] > 0:
        Q = apply_A(P)
        PtQ = P.T @ Q
        alpha = np.linalg.solve(PtQ, P.T @ R)
        X = X + P @ alpha
        R = R - Q @ alpha
        it += 1
        hist.append(float(np.max(np.linalg.norm(R, axis=0) / bn)))
        if hist[-1] <= tol:
            break
        Z = apply_M(R)
        beta = -np.linalg.solve(PtQ, Q.T @ Z)
        P = orth(Z + P @ beta, drop_tol)
    return X, it, hist


# ----------------------------------------------------------------------------------------
# Algorithm 2 steps 5-10 (Algorithm 1 steps 3-8): Nyström core
# ----------------------------------------------------------------------------------------
def nystrom_core(G, Y, k, eps_rel=1e-10):
    """Returns (U_k, Sigma_k, info).

    Y = B G. Steps: Y = QR (step 5); C = G^T Y (step 6, symmetrized: the paper is silent,
    C is symmetric in exact arithmetic); EVD C, keep eigenvalues >= eps (step 7; eps taken
    relative to the largest eigenvalue, non-positive ones always dropped);
    T = R V1 D1^{-1} V1^T R^T (step 8); EVD T = W E W^T, descending (step 9);
    U = Q W(:, 1:k), Sigma = E(1:k) (step 10; Y there is the Q of step 5).
    The rank is min(r, k) with r the number of kept eigenvalues of C (§2.1).
    """
    Q, R = np.linalg.qr(Y)                     # step 5
    C = G.T @ Y                                # step 6
    C = 0.5 * (C + C.T)
    d, V = np.linalg.eigh(C)                   # step 7
    dmax = d.max() if d.size else 0.0
    keep = d >= max(eps_rel * dmax, np.finfo(np.float64).tiny)
    V1, D1 = V[:, keep], d[keep]
    RV1 = R @ V1
    T = (RV1 / D1) @ RV1.T                     # step 8
    T = 0.5 * (T + T.T)
    e, W = np.linalg.eigh(T)                   # step 9
    order = np.argsort(e)[::-1]
    e, W = e[order], W[:, order]
    r = int(keep.sum())
    kk = min(k, r)
    U = Q @ W[:, :kk]                          # step 10
    return U, e[:kk], dict(rank_C=r, eig_C=d, eig_T=e)


class M2:
    """M2 = A_Gamma^{-1} + Z Sigma Z^T (§4.3 eq. (left_prec_mat), Algorithm 2 step 12)."""

    def __init__(self, dbbd, Z, Sigma):
        self.dbbd, self.Z, self.Sigma = dbbd, Z, Sigma

    def apply(self, r):
        return self.dbbd.solve_G(r) + self.Z @ (self.Sigma[:, None] * (self.Z.T @ r)
                                               if np.ndim(r) == 2 else self.Sigma * (self.Z.T @ r))

    def dense(self):
        n = self.dbbd.n_G
        return self.dbbd.solve_G(np.eye(n)) + (self.Z * self.Sigma) @ self.Z.T


class M2ADEF:
    """M_{2A-DEF}, the adapted-deflation variant of M2 (§4.3).

    §4.3 defines, for a basis Ub of the R_G-transformed space, E = Ub^T R_G^{-T} S_G R_G^{-1} Ub,
    Q = Ub E^{-1} Ub^T, the deflation operator I - Q R_G^{-T} S_G R_G^{-1} + Q (eq.
    (deflation_comp_from_low_rank)) and the preconditioner R_G^{-1} (.) R_G^{-T} (eq.
    (our_two_level_preconditioner)); M_{2A-DEF} is the same construction on the M2
    approximation A_GI S_I^{-1} A_IG ~ U Sigma U^T, whose transformed basis is R_G^{-T} U.
    With Zk = R_G^{-1} R_G^{-T} U = A_G^{-1} U (Algorithm 2 step 11) every R_G cancels:
        E = Zk^T S_G Zk,   M = A_G^{-1} - Zk E^{-1} Zk^T S_G A_G^{-1} + Zk E^{-1} Zk^T.
    Sigma does not enter (Q is invariant under a change of basis of span(Zk)). A column of
    Zk that is (numerically) in the span of the others is left out by the thresholded
    Cholesky rule of ``kept_columns`` applied to E, which leaves span(Zk), hence Q, unchanged.
    """

    def __init__(self, dbbd, Zk, Sigma=None, drop_tol=1e-12):
        self.dbbd, self.Sigma = dbbd, Sigma
        Z = np.asarray(Zk, dtype=np.float64)
        E = Z.T @ dbbd.apply_S_gamma(Z)
        E = 0.5 * (E + E.T)
        keep = kept_columns(E, drop_tol)
        self.Z, self.E = Z[:, keep], E[np.ix_(keep, keep)]
        self._Ec = sla.cho_factor(self.E, lower=True)

    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        y = self.dbbd.solve_G(r)                               # A_G^{-1} r
        Sy = self.dbbd.apply_S_gamma(y)                        # S_G A_G^{-1} r
        c = sla.cho_solve(self._Ec, self.Z.T @ r - self.Z.T @ Sy)
        return y + self.Z @ c

    def dense(self):
        n = self.dbbd.n_G
        return self.apply(np.eye(n))


def sketch_product(dbbd, G, eps_inner=0.1, form="S_gamma", maxit=500, drop_tol=1e-12):
    """Algorithm 2 steps 2-4: Y = A_GI S_I^{-1} A_IG G through the inner block PCG.
    Returns (X, Y, iterations, residual history); the forms are those of build_m2."""
    if form == "S_I":
        F = dbbd.A_IG @ G
        X, it, hist = block_pcg(dbbd.apply_S_I, dbbd.solve_I, F, eps_inner, maxit, drop_tol)
        Y = dbbd.A_GI @ X
    elif form == "S_gamma":
        Fh = dbbd.A_GI @ dbbd.solve_I(dbbd.A_IG @ G)
        X, it, hist = block_pcg(dbbd.apply_S_gamma, dbbd.solve_G, Fh, eps_inner, maxit,
                                drop_tol)
        Y = dbbd.A_G @ X
    elif form == "S_gamma_naive":
        AG = dbbd.A_G @ G
        X, it, hist = block_pcg(dbbd.apply_S_gamma, dbbd.solve_G, AG, eps_inner, maxit,
                                drop_tol)
        Y = dbbd.A_G @ X - AG
    else:
        raise ValueError(form)
    return X, Y, it, hist


def build_m2(dbbd, G, k, eps_inner=0.1, form="S_gamma", eps_rel=1e-10, maxit=500,
             drop_tol=1e-12, variant="M2", q=0):
    """Algorithm 2. Returns (M2, info); variant="M2_ADEF" returns M_{2A-DEF} (class
    M2ADEF) built from the same Z = A_G^{-1} U.

    q > 0: the q-power iteration Nyström method of §2.1 eq. (power), G = B^q Omega with
    B = A_GI S_I^{-1} A_IG and Omega the given sketch, the columns orthonormalized after
    every application of B (thresholded Cholesky-QR ``orth``; a column that falls in the
    span of the others is dropped). Each application of B is one inner block PCG (steps 2-4)
    and the last one gives the Y of step 4 for the final G.

    form="S_I":     F = A_IG G (step 2); solve S_I X = F by block PCG preconditioned by
                    A_I (step 3, §5 setup); Y = A_GI X (step 4).
    form="S_gamma": the same Y through the interface Schur complement. With
                    T = A_GI A_I^{-1} A_IG (so S_Gamma = A_G - T) and the SMW
                    identity (§4.1 eq. (S-1)), A_G S_Gamma^{-1} T = A_G S_Gamma^{-1} A_G - A_G
                    = A_GI S_I^{-1} A_IG. So: Fh = T G; solve S_Gamma E = Fh by block PCG
                    preconditioned by A_G (the first level S1, §2.3 eq. (S1)); Y = A_G E.
    form="S_gamma_naive": solve S_Gamma Xh = A_G G, Y = A_G Xh - A_G G (same Y for exact
                    solves, but the relative tolerance is measured against the trivial part
                    A_G G of the right-hand side, so a loose tolerance stops too early).
    """
    G = np.asarray(G, dtype=np.float64)
    it_power = []
    for _ in range(q):                                    # eq. (power)
        _, Yq, itq, _ = sketch_product(dbbd, G, eps_inner, form, maxit, drop_tol)
        it_power.append(itq)
        G = orth(Yq, drop_tol)
    X, Y, it, hist = sketch_product(dbbd, G, eps_inner, form, maxit, drop_tol)
    U, Sigma, info = nystrom_core(G, Y, k, eps_rel)       # steps 5-10
    Z = dbbd.solve_G(U)                                   # step 11
    info.update(it_inner=it, inner_hist=hist, X=X, Y=Y, U=U, G=G, it_power=it_power)
    if variant == "M2_ADEF":
        return M2ADEF(dbbd, Z, Sigma, drop_tol), info
    if variant != "M2":
        raise ValueError(variant)
    return M2(dbbd, Z, Sigma), info


def build_m1(dbbd, G, k, eps_inner=0.1, form="S_gamma", eps_rel=1e-10, maxit=500,
             drop_tol=1e-12):
    """The variant M1 of §4.1 (eq. (proposed_deflation_prec), eq. (prec1S)).

    R_G is the dense upper Cholesky factor of A_G (A_G = R^T R), so this is for interfaces of
    up to a few thousand unknowns. Nyström (Algorithm 1) of
    B = R^{-T} A_GI S_I^{-1} A_IG R^{-1} (eq. (lr_approximation_S-1_A-I)) with the sketch G:
    F = B G = R^{-T} Y, where Y = A_GI S_I^{-1} A_IG (R^{-1} G) comes from the inner block PCG
    (steps 2-4 of Algorithm 2 on the sketch R^{-1} G); steps 3-8 of Algorithm 1 on (G, F) give
    Ub, Sigma; Zb = R^{-1} Ub and M1 = A_G^{-1} + Zb Sigma Zb^T. Returns (M1, info).
    """
    G = np.asarray(G, dtype=np.float64)
    R = np.linalg.cholesky(dbbd.A_G.toarray()).T
    Gp = sla.solve_triangular(R, G, lower=False)                  # R^{-1} G
    X, Y, it, hist = sketch_product(dbbd, Gp, eps_inner, form, maxit, drop_tol)
    F = sla.solve_triangular(R, Y, trans="T", lower=False)        # R^{-T} Y
    Ub, Sigma, info = nystrom_core(G, F, k, eps_rel)
    Zb = sla.solve_triangular(R, Ub, lower=False)                 # R^{-1} Ub
    info.update(it_inner=it, inner_hist=hist, X=X, Y=Y, U=Ub, R=R)
    return M2(dbbd, Zb, Sigma), info


def build_m3(dbbd, G_I, k, eps_inner=0.1, eps_rel=1e-10, maxit=500, drop_tol=1e-12,
             variant="M3"):
    """The variant M3 of §4.3 (eq. (internal_term_lr_approximation_2), eq. (left_prec_mat2)).

    Nyström (Algorithm 1) applied to B = S_I^{-1} with the sketch G_I (n_I x (k+p)):
    F = S_I^{-1} G_I by block PCG on S_I X = G_I preconditioned by A_I (the inner solver of
    §5), then steps 3-8 of Algorithm 1 give S_I^{-1} ~ V Sigma V^T; Zh = A_G^{-1} A_GI V and
    M3 = A_G^{-1} + Zh Sigma Zh^T. variant="M3_ADEF" deflates span(Zh) instead, like
    M_{2A-DEF} (class M2ADEF). Returns (preconditioner, info).
    """
    G_I = np.asarray(G_I, dtype=np.float64)
    X, it, hist = block_pcg(dbbd.apply_S_I, dbbd.solve_I, G_I, eps_inner, maxit, drop_tol)
    V, Sigma, info = nystrom_core(G_I, X, k, eps_rel)
    Zh = dbbd.solve_G(dbbd.A_GI @ V)
    info.update(it_inner=it, inner_hist=hist, X=X, V=V)
    if variant == "M3_ADEF":
        return M2ADEF(dbbd, Zh, Sigma, drop_tol), info
    if variant != "M3":
        raise ValueError(variant)
    return M2(dbbd, Zh, Sigma), info


# ----------------------------------------------------------------------------------------
# Recursive treatment of A_Gamma (concluding section: the systems with A_Gamma replaced by
# systems with a much smaller matrix). Reading: A_Gamma gets a DBBD split of its own (§2.3
# eq. (perm_A) applied to A_Gamma, interior blocks C_i and a second-level interface Gamma_2),
# and A_Gamma^{-1} is replaced by the block elimination of §2.3 eq. (A_LDLT) for that split
# whose Schur-complement solve is the two-level preconditioner M2 of that split (Algorithm 2
# on A_Gamma). Only C_i and C_Gamma_2 are factorized.
# ----------------------------------------------------------------------------------------
class NestedGammaInverse:
    """x = A_Gamma~^{-1} b for A_Gamma = [[C_I, C_IG2], [C_G2I, C_G2]] (rows of A_Gamma split by
    the DBBD ``d2``): y = C_I^{-1} b_I, x_G2 = M2' (b_G2 - C_G2I y), x_I = C_I^{-1} (b_I - C_IG2
    x_G2), with M2' the two-level preconditioner of S_C = C_G2 - C_G2I C_I^{-1} C_IG2. It is
    A_Gamma^{-1} exactly when M2' = S_C^{-1}."""

    def __init__(self, d2, m2):
        self.d2, self.m2 = d2, m2

    def apply(self, B):
        d2 = self.d2
        B = np.asarray(B, dtype=np.float64)
        bI, bG = B[d2.interior], B[d2.gamma]
        y = d2.solve_I(bI)
        xG = self.m2.apply(bG - d2.A_GI @ y)
        xI = d2.solve_I(bI - d2.A_IG @ xG)
        X = np.empty_like(B)
        X[d2.interior] = xI
        X[d2.gamma] = xG
        return X


def recursive_gamma(dbbd, part2, nblocks2, G2, k2, eps_inner=0.1, eps_rel=1e-10, maxit=500,
                    drop_tol=1e-12):
    """The DBBD ``dbbd`` with A_Gamma^{-1} replaced by the nested two-level inverse.

    part2: DBBD partition of A_Gamma (rows in dbbd.gamma order; labels in [0, nblocks2) or
    -1 for Gamma_2); G2: the nested sketch (n_Gamma_2 x (k2 + p2), Gamma_2 unknowns in
    increasing row order of A_Gamma). Algorithm 2 runs on A_Gamma's split (S_Gamma form).
    Returns (dbbd', info): dbbd' is a shallow copy whose solve_G applies the nested inverse
    (apply_S_gamma is unchanged: S_Gamma stays exact); build_m2(dbbd', ...) is then the
    recursive M2 = A_Gamma~^{-1} + Z Sigma Z^T with Z = A_Gamma~^{-1} U, and
    solve(dbbd', ...) its outer PCG. Only the S_Gamma inner form is meant for dbbd'.
    """
    import copy
    d2 = DBBD(dbbd.A_G, part2, nblocks2)
    m2, info2 = build_m2(d2, G2, k2, eps_inner, "S_gamma", eps_rel, maxit, drop_tol)
    inv = NestedGammaInverse(d2, m2)
    out = copy.copy(dbbd)
    out.solve_G = inv.apply
    return out, dict(d2=d2, m2=m2, inverse=inv, it_inner=info2["it_inner"], info=info2)


# ----------------------------------------------------------------------------------------
# Outer PCG on S_Gamma w = f (§2.3 eq. (Sx=b)), and the block elimination of §2.3 eq. (A_LDLT)
# ----------------------------------------------------------------------------------------
def pcg(apply_A, apply_M, f, rtol=1e-8, maxit=500, x0=None, coeffs=None):
    """Textbook PCG. Stops when ||r_k|| / ||f|| <= rtol on the updated residual.

    Returns (x, iterations, residual history); iterations = number of operator applies.
    ``coeffs`` (a dict, optional) receives the step lengths alpha_j = r_j^T z_j / p_j^T A p_j
    ("alpha", one per iteration) and the ratios beta_j = r_{j+1}^T z_{j+1} / r_j^T z_j that
    formed the next direction ("beta", one fewer).
    """
    f = np.asarray(f, dtype=np.float64)
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    r = f - apply_A(x) if x0 is not None else f.copy()
    fn = np.linalg.norm(f)
    if fn == 0.0:
        return x, 0, [0.0]
    hist = [np.linalg.norm(r) / fn]
    if hist[-1] <= rtol:
        return x, 0, hist
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    if coeffs is not None:
        coeffs["alpha"], coeffs["beta"] = [], []
    while it < maxit:
        q = apply_A(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / fn)
        if coeffs is not None:
            coeffs["alpha"].append(float(alpha))
        if hist[-1] <= rtol:
            break
        z = apply_M(r)
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        if coeffs is not None:
            coeffs["beta"].append(float(beta))
    return x, it, hist


def lanczos_tridiagonal(alpha, beta):
    """The m x m Lanczos tridiagonal T of PCG's first m iterations (Saad, Iterative Methods
    for Sparse Linear Systems, 2nd ed., §6.7.3: CG and Lanczos generate the same Krylov
    basis). With preconditioner M and operator A, T is the matrix of the symmetrized
    operator M^{1/2} A M^{1/2} in the orthonormal basis of normalized preconditioned
    residuals; written in the coefficients alone:
        T[0, 0] = 1 / alpha_0,
        T[j, j] = 1 / alpha_j + beta_{j-1} / alpha_{j-1}          (j >= 1),
        T[j-1, j] = T[j, j-1] = sqrt(beta_{j-1}) / alpha_{j-1}.
    Its eigenvalues are Ritz values of the preconditioned operator M A; after n steps on an
    n x n system they are its eigenvalues."""
    a = np.asarray(alpha, dtype=np.float64)
    b = np.asarray(beta, dtype=np.float64)[:max(len(a) - 1, 0)]
    m = len(a)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / a[j] + (b[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j > 0:
            T[j - 1, j] = T[j, j - 1] = np.sqrt(b[j - 1]) / a[j - 1]
    return T


def kappa_estimate(alpha, beta):
    """(lambda_min, lambda_max, kappa) of the preconditioned operator estimated by the
    extreme eigenvalues of ``lanczos_tridiagonal`` (numpy's symmetric EVD as one step)."""
    if len(alpha) == 0:
        return 0.0, 0.0, 0.0
    e = np.linalg.eigvalsh(lanczos_tridiagonal(alpha, beta))
    return float(e[0]), float(e[-1]), float(e[-1] / e[0])


def solve(dbbd, prec_apply, b, rtol=1e-8, maxit=500, coeffs=None):
    """x = A^{-1} b by the block elimination of §2.3 eq. (A_LDLT) with PCG on S_Gamma (§2.3 eq. (Sx=b)).

    f = b_G - A_GI A_I^{-1} b_I; PCG on S_Gamma w = f preconditioned by ``prec_apply``;
    x_G = w, x_I = A_I^{-1}(b_I - A_IG w). Returns (x, it_PCG, history).
    """
    b = np.asarray(b, dtype=np.float64)
    bI, bG = b[dbbd.interior], b[dbbd.gamma]
    f = bG - dbbd.A_GI @ dbbd.solve_I(bI)
    w, it, hist = pcg(dbbd.apply_S_gamma, prec_apply, f, rtol, maxit, coeffs=coeffs)
    xI = dbbd.solve_I(bI - dbbd.A_IG @ w)
    x = np.empty(dbbd.n)
    x[dbbd.interior] = xI
    x[dbbd.gamma] = w
    return x, it, hist


def solve_full_space(dbbd, prec_apply, b, rtol=1e-8, maxit=500, coeffs=None):
    """PCG on A x = b with the block-factorization preconditioner of §2.3 (Schur block M2).

    M^{-1} r: z_G = M2 (r_G - A_GI A_I^{-1} r_I), z_I = A_I^{-1}(r_I - A_IG z_G).
    Start x0 = (A_I^{-1} b_I, 0), so r0 = (0, f). While r_I = 0 the iterates coincide with
    PCG on S_Gamma w = f preconditioned by M2 (z_I = -A_I^{-1} A_IG z_G gives A z = (0,
    S_Gamma z_G)); stopping uses ||r|| / ||f|| with f the interface part of r0.
    """
    b = np.asarray(b, dtype=np.float64)
    I, Gm = dbbd.interior, dbbd.gamma
    A = dbbd.A

    def prec(r):
        rI, rG = r[I], r[Gm]
        zG = prec_apply(rG - dbbd.A_GI @ dbbd.solve_I(rI))
        zI = dbbd.solve_I(rI - dbbd.A_IG @ zG)
        z = np.empty_like(r)
        z[I], z[Gm] = zI, zG
        return z

    x0 = np.zeros(dbbd.n)
    x0[I] = dbbd.solve_I(b[I])
    r0 = b - A @ x0
    fn = np.linalg.norm(r0)
    x, it, hist = pcg(lambda v: A @ v, prec, r0, rtol, maxit, coeffs=coeffs)
    return x0 + x, it, hist


def relative_residual(A, x, b):
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))
