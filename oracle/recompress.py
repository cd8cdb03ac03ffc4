"""Algebraic recompression of the interpolation H2 approximation.

TEST INFRASTRUCTURE ONLY (part of the oracle): plain numpy in FP64, loops over
clusters and blocks; nothing on the product path imports it.

The paper reaches its storage figures with an H2 matrix whose cluster bases
are compressed algebraically, "without a significant loss of accuracy"
(Section "H2-Matrix Compression", the recompression step after the
hybrid cross approximation).  The steps here follow the published algorithms
for nested bases (S. Boerm, Efficient Numerical Methods for Non-local
Operators, EMS 2010, chapters on orthogonalisation and on the compression of
H2 matrices with total cluster-basis weights), applied to the direct
Chebyshev-interpolation H2 of ``H2Oracle``:

1. Nested form: leaf bases V_t, W_t and transfer matrices
   E_c(nu', nu) = L^parent_nu(x^c_nu') (interpolation reproduces the parent's
   polynomials, so V_parent|c = V_c E_c exactly), couplings S_ts.
2. Orthogonalisation, leaves to root: V_t = Q_t R_t (QR); a parent stacks its
   children's R_c E_c and factorises again, which gives orthonormal nested
   bases Q_t with transfers Qhat_c, and S'_ts = R_t S_ts T_s^T.
3. Total weights, root to leaves: the far-field rows of t in Q_t coordinates
   are spanned by [S'_ts for the blocks of t, Qhat_t Z_parent] (the
   ancestors' blocks reach t through the transfers); Z_t is that matrix
   condensed to at most k_t columns with the same Gram matrix.
4. Truncation, leaves to root: the leading left singular vectors X_t of the
   weight (for a parent: the weight expressed in its children's new bases,
   G_t Z_t with G_t = [B_c Qhat_c]) whose singular values exceed
   ``eps`` times the largest; the new transfers are the children's rows of
   X_t and B_t = X_t^T G_t maps old coordinates to new ones.
5. New couplings B_t S'_ts B'_s^T.

The same is done for the column bases (W, with the blocks' transposes).
"""
from __future__ import annotations

import numpy as np

from . import cheb_points, lagrange3


def _tree_order(tree):
    """Clusters sorted by level: (root first, leaves last)."""
    return np.argsort(tree["level"], kind="stable")


def nested_form(h):
    """Leaf bases, transfers and couplings of an ``H2Oracle`` (store=True)."""
    t = h.tree()
    b = h.blocks()
    nc = h.n_clusters
    leaf = t["child0"] < 0
    V, W, E = {}, {}, {}
    for c in range(nc):
        if leaf[c]:
            V[c], W[c] = h.cluster_bases(c, int(t["size"][c]))
        p = t["parent"][c]
        if p >= 0:
            pts = cheb_points(t["box"][c], h.m)
            E[c] = np.array([lagrange3(t["box"][p], h.m, x)[0] for x in pts])
    S = {(int(a), int(s)): h.coupling(int(a), int(s)) for a, s in zip(b["far_t"], b["far_s"])}
    return {"tree": t, "leaf": leaf, "V": V, "W": W, "E": E, "S": S, "k": h.k, "nc": nc}


def _orthogonalise(form, leaf_bases):
    """Q (leaves), Qhat (transfers of every non-root cluster) and R."""
    t, leaf = form["tree"], form["leaf"]
    Q, Qhat, R = {}, {}, {}
    for c in _tree_order(t)[::-1]:
        c = int(c)
        if leaf[c]:
            Q[c], R[c] = np.linalg.qr(leaf_bases[c])
        else:
            c0, c1 = int(t["child0"][c]), int(t["child1"][c])
            M = np.vstack([R[c0] @ form["E"][c0], R[c1] @ form["E"][c1]])
            Qh, R[c] = np.linalg.qr(M)
            n0 = R[c0].shape[0]
            Qhat[c0], Qhat[c1] = Qh[:n0], Qh[n0:]
    return Q, Qhat, R


def _condense(Y, rows):
    """A matrix with at most `rows` columns and the Gram matrix Y Y^T."""
    if Y.shape[1] <= rows:
        return Y
    _, Rf = np.linalg.qr(Y.T)
    return Rf.T


def _weights(form, Qhat, R, blocks_of, coupling):
    """Total weights Z_t, root to leaves (``coupling(c, other)`` in Q coords)."""
    t = form["tree"]
    Z = {}
    for c in _tree_order(t):
        c = int(c)
        kc = R[c].shape[0]
        cols = [coupling(c, o) for o in blocks_of[c]]
        p = int(t["parent"][c])
        if p >= 0 and Z[p].shape[1] > 0:
            cols.append(Qhat[c] @ Z[p])
        Z[c] = _condense(np.hstack(cols), kc) if cols else np.zeros((kc, 0))
    return Z


def _truncate(form, Q, Qhat, Z, eps):
    """New leaf bases, transfers and the old-to-new coordinate maps B_t."""
    t, leaf = form["tree"], form["leaf"]
    Qn, En, B, rank = {}, {}, {}, {}
    for c in _tree_order(t)[::-1]:
        c = int(c)
        if leaf[c]:
            G = np.eye(Q[c].shape[1])
        else:
            c0, c1 = int(t["child0"][c]), int(t["child1"][c])
            G = np.vstack([B[c0] @ Qhat[c0], B[c1] @ Qhat[c1]])
        Wt = G @ Z[c]
        if Wt.shape[1] == 0 or Wt.shape[0] == 0:
            X = np.zeros((G.shape[0], 0))
        else:
            U, sv, _ = np.linalg.svd(Wt, full_matrices=False)
            keep = int(np.sum(sv > eps * sv[0])) if sv[0] > 0 else 0
            X = U[:, :keep]
        rank[c] = X.shape[1]
        B[c] = X.T @ G
        if leaf[c]:
            Qn[c] = Q[c] @ X
        else:
            n0 = B[c0].shape[0]
            En[c0], En[c1] = X[:n0], X[n0:]
    return Qn, En, B, rank


def recompress(h, eps: float, form: dict | None = None) -> dict:
    """Recompressed H2 form of an ``H2Oracle`` at relative truncation ``eps``
    (``eps = 0``: orthogonalisation only, every nonzero direction kept);
    ``form``: the nested form of ``h`` if already built."""
    form = form if form is not None else nested_form(h)
    nc = form["nc"]
    far_by_t = {c: [] for c in range(nc)}
    far_by_s = {c: [] for c in range(nc)}
    for (a, s) in form["S"]:
        far_by_t[a].append(s)
        far_by_s[s].append(a)
    Qr, Qhr, Rr = _orthogonalise(form, form["V"])
    Qc, Qhc, Rc = _orthogonalise(form, form["W"])
    Sp = {(a, s): Rr[a] @ S @ Rc[s].T for (a, s), S in form["S"].items()}
    Zr = _weights(form, Qhr, Rr, far_by_t, lambda c, o: Sp[(c, o)])
    Zc = _weights(form, Qhc, Rc, far_by_s, lambda c, o: Sp[(o, c)].T)
    Vn, En, Br, rank_r = _truncate(form, Qr, Qhr, Zr, eps)
    Wn, Fn, Bc, rank_c = _truncate(form, Qc, Qhc, Zc, eps)
    Sn = {(a, s): Br[a] @ S @ Bc[s].T for (a, s), S in Sp.items()}
    return {"tree": form["tree"], "leaf": form["leaf"], "V": Vn, "W": Wn, "E": En, "F": Fn,
            "S": Sn, "rank_row": rank_r, "rank_col": rank_c, "k": form["k"], "form": form}


def far_matvec_direct(h, x) -> np.ndarray:
    """sum over far blocks of V_t S_ts W_s^T x|_s with the direct bases."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    t, b = h.tree(), h.blocks()
    bases = {}

    def basis(c):
        if c not in bases:
            bases[c] = h.cluster_bases(c, int(t["size"][c]))
        return bases[c]

    y = np.zeros_like(x)
    for a, s in zip(b["far_t"], b["far_s"]):
        a, s = int(a), int(s)
        ti = t["perm"][t["start"][a]:t["start"][a] + t["size"][a]]
        si = t["perm"][t["start"][s]:t["start"][s] + t["size"][s]]
        y[:, ti] += ((basis(a)[0] @ h.coupling(a, s)) @ (basis(s)[1].T @ x[:, si].T)).T
    return y


def far_matvec(rc: dict, x) -> np.ndarray:
    """The far field of a recompressed form: upward, coupling, downward."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    t, leaf = rc["tree"], rc["leaf"]
    order = _tree_order(t)
    xh, yh = {}, {}
    for c in order[::-1]:
        c = int(c)
        if leaf[c]:
            si = t["perm"][t["start"][c]:t["start"][c] + t["size"][c]]
            xh[c] = rc["W"][c].T @ x[:, si].T
        else:
            c0, c1 = int(t["child0"][c]), int(t["child1"][c])
            xh[c] = rc["F"][c0].T @ xh[c0] + rc["F"][c1].T @ xh[c1]
        yh[c] = np.zeros((rc["rank_row"][c], x.shape[0]))
    for (a, s), S in rc["S"].items():
        yh[a] += S @ xh[s]
    y = np.zeros_like(x)
    for c in order:
        c = int(c)
        if leaf[c]:
            ti = t["perm"][t["start"][c]:t["start"][c] + t["size"][c]]
            y[:, ti] += (rc["V"][c] @ yh[c]).T
        else:
            for ch in (int(t["child0"][c]), int(t["child1"][c])):
                yh[ch] += rc["E"][ch] @ yh[c]
    return y


def matvec(h, rc: dict, x) -> np.ndarray:
    """The H2 product with the recompressed far field and the exact near field."""
    return h.matvec(x) - far_matvec_direct(h, x) + far_matvec(rc, x)


def storage(rc: dict) -> dict:
    """Stored coefficients before (interpolation, rank k everywhere; one copy
    of each transfer per side) and after recompression."""
    t, leaf, k = rc["tree"], rc["leaf"], rc["k"]
    nonroot = [c for c in range(len(leaf)) if t["parent"][c] >= 0]
    before = {"bases": int(sum(2 * int(t["size"][c]) * k for c in range(len(leaf)) if leaf[c])),
              "transfers": 2 * k * k * len(nonroot),
              "coupling": k * k * len(rc["S"])}
    rr, rcol = rc["rank_row"], rc["rank_col"]
    after = {"bases": int(sum(int(t["size"][c]) * (rr[c] + rcol[c]) for c in range(len(leaf)) if leaf[c])),
             "transfers": int(sum(rr[c] * rr[int(t["parent"][c])] + rcol[c] * rcol[int(t["parent"][c])]
                                  for c in nonroot)),
             "coupling": int(sum(rr[a] * rcol[s] for (a, s) in rc["S"]))}
    before["total"] = sum(before.values())
    after["total"] = sum(after.values())
    return {"before": before, "after": after}
