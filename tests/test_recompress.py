"""Oracle of the algebraic H2 recompression (oracle/recompress.py).

Pins: with no truncation the orthogonalised nested form reproduces the
interpolation far field to rounding and its bases are orthonormal and nested;
with truncation the error against the interpolation H2 product follows the
relative threshold, the stored coefficients fall as it grows, and the product
stays as close to the dense operator as the interpolation H2 itself.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import recompress as rcm


@pytest.fixture(scope="module")
def case():
    m = synth.icosphere(3)
    h = oracle.H2Oracle(m.xyz, m.tri, 4, 16, 2.0)
    form = rcm.nested_form(h)
    x = synth.gaussian_rhs(m.n_vertices, 2, 3)
    return m, h, form, x


def _full_basis(rc, c):
    """The recompressed row basis of cluster c on its own rows (tree order)."""
    t = rc["tree"]
    if rc["leaf"][c]:
        return rc["V"][c]
    c0, c1 = int(t["child0"][c]), int(t["child1"][c])
    return np.vstack([_full_basis(rc, c0) @ rc["E"][c0], _full_basis(rc, c1) @ rc["E"][c1]])


def test_orthogonalised_form_reproduces_the_far_field(case):
    m, h, form, x = case
    rc = rcm.recompress(h, 0.0, form)
    yd = rcm.far_matvec_direct(h, x)
    yr = rcm.far_matvec(rc, x)
    assert np.linalg.norm(yr - yd) <= 1e-12 * np.linalg.norm(yd)
    t = rc["tree"]
    checked = 0
    for c in range(h.n_clusters):
        if rc["rank_row"][c] == 0 or t["size"][c] > 200:
            continue
        Q = _full_basis(rc, c)
        assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
        checked += 1
    assert checked > 10


def test_truncation_follows_the_threshold(case):
    m, h, form, x = case
    y = h.matvec(x)
    errs, sizes = [], []
    for eps in (1e-8, 1e-6, 1e-4, 1e-2):
        rc = rcm.recompress(h, eps, form)
        errs.append(np.linalg.norm(rcm.matvec(h, rc, x) - y) / np.linalg.norm(y))
        sizes.append(rcm.storage(rc)["after"]["total"])
        assert errs[-1] <= 0.2 * eps, (eps, errs[-1])
    assert all(a < b for a, b in zip(errs, errs[1:])), errs
    assert all(a > b for a, b in zip(sizes, sizes[1:])), sizes


def test_recompressed_product_stays_at_the_interpolation_error(case):
    m, h, form, x = case
    M = oracle.dense_matrix(m.xyz, m.tri)
    yd = (M @ x.T).T
    e_h2 = np.linalg.norm(h.matvec(x) - yd) / np.linalg.norm(yd)
    rc = rcm.recompress(h, 1e-6, form)
    e_rc = np.linalg.norm(rcm.matvec(h, rc, x) - yd) / np.linalg.norm(yd)
    assert e_rc <= 1.01 * e_h2
    st = rcm.storage(rc)
    assert st["after"]["coupling"] < 0.5 * st["before"]["coupling"]
    assert max(rc["rank_row"].values()) <= h.k and max(rc["rank_col"].values()) <= h.k


def _leaf_block_row(h, leaf, bases):
    """The far field on the rows of leaf `leaf`: every admissible block (a, s)
    whose target `a` contains the leaf, from the direct bases, as a |leaf| x N
    matrix (mesh-ordered columns)."""
    tr, b = h.tree(), h.blocks()
    n0, n = int(tr["start"][leaf]), int(tr["size"][leaf])
    K = np.zeros((n, h.N))
    for a, s in zip(b["far_t"], b["far_s"]):
        a, s = int(a), int(s)
        a0, an = int(tr["start"][a]), int(tr["size"][a])
        if not (a0 <= n0 and n0 + n <= a0 + an):
            continue
        V = bases(a)[0][n0 - a0:n0 - a0 + n]
        si = tr["perm"][tr["start"][s]:tr["start"][s] + tr["size"][s]]
        K[:, si] += V @ h.coupling(a, s) @ bases(s)[1].T
    return K


def test_leaf_bases_keep_the_total_block_row_to_the_threshold(case):
    """At a leaf the truncation is the SVD of the total weight, which carries
    the blocks of the leaf and of all its ancestors: projecting the leaf's whole
    far-field block row onto the new basis loses at most eps times its norm.
    (A weight that left out the ancestors' blocks would not.)"""
    m, h, form, x = case
    eps = 1e-4
    rc = rcm.recompress(h, eps, form)
    tr = h.tree()
    cache = {}

    def bases(c):
        if c not in cache:
            cache[c] = h.cluster_bases(c, int(tr["size"][c]))
        return cache[c]

    leaves = [c for c in range(h.n_clusters) if rc["leaf"][c] and rc["rank_row"][c] > 0]
    worst = 0.0
    for c in leaves[::max(1, len(leaves) // 12)]:
        K = _leaf_block_row(h, c, bases)
        Q = rc["V"][c]
        lost = np.linalg.norm(K - Q @ (Q.T @ K), 2) / np.linalg.norm(K, 2)
        worst = max(worst, lost)
    assert worst <= eps * (1 + 1e-6), worst
    assert worst > 0.0
