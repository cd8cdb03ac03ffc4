"""Where the reduced forms' error budgets come from, on the oracle (CPU).

The reduced forms store the far-field matrices in FP32 or as BF16 pairs
hi = bf16(a), lo = bf16(a - hi) (relative representation error <= 2^-17)
and keep the near field, the diagonal and the final sums in FP64.  Rounding
only the stored coupling matrices S_ts (the bulk of the far field) and the
leaf bases of the oracle's H2 operator, and multiplying in FP64, isolates the
storage part of their error.  Measured on an icosphere of level 4 (m = 4):
FP32 1.5e-8, far inside the 1e-5 budget; BF16 pairs 7.1e-7, some 2^5.5 times
higher (17 bits against 24, partly averaged out in the sums), still inside it;
one BF16 word alone (8 bits) 5e-4, outside it, which is why the pairs are
stored.  The BF16 form's GPU error (2.7e-5 to 8.6e-5 on the benchmark meshes)
adds the rounding of the vectors and transfers and the FP32 accumulation,
hence its 1e-4 budget.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import recompress as rcm


def bf16(a):
    """Round-to-nearest-even FP32 -> BF16 (kept in an FP32 container)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    u = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return u.view(np.float32)


def bf16_pair(a):
    a32 = np.asarray(a, dtype=np.float64)
    hi = bf16(a32.astype(np.float32)).astype(np.float64)
    lo = bf16((a32 - hi).astype(np.float32)).astype(np.float64)
    return hi + lo


def far_field(h, x, round_s, round_vw):
    t, b = h.tree(), h.blocks()
    cache = {}

    def bases(c):
        if c not in cache:
            V, W = h.cluster_bases(c, int(t["size"][c]))
            cache[c] = (round_vw(V), round_vw(W))
        return cache[c]

    y = np.zeros_like(x)
    for a, s in zip(b["far_t"], b["far_s"]):
        a, s = int(a), int(s)
        ti = t["perm"][t["start"][a]:t["start"][a] + t["size"][a]]
        si = t["perm"][t["start"][s]:t["start"][s] + t["size"][s]]
        y[:, ti] += ((bases(a)[0] @ round_s(h.coupling(a, s))) @ (bases(s)[1].T @ x[:, si].T)).T
    return y


@pytest.fixture(scope="module")
def case():
    m = synth.icosphere(4)
    h = oracle.H2Oracle(m.xyz, m.tri, 4, 32, 2.0)
    x = synth.gaussian_rhs(m.n_vertices, 2, 8)
    return h, x, h.matvec(x), rcm.far_matvec_direct(h, x)


def test_bf16_pair_keeps_17_bits():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(100000) * 10.0 ** rng.uniform(-6, 3, 100000)
    rel = np.abs(bf16_pair(a) - a) / np.abs(a)
    assert np.max(rel) <= 2.0 ** -17 * (1 + 1e-6)
    assert np.max(np.abs(bf16(a.astype(np.float32)) - a) / np.abs(a)) > 2.0 ** -10   # one BF16 alone: 8 bits


def test_storage_error_of_the_reduced_forms(case):
    h, x, y, yfar = case

    def err(round_s, round_vw):
        yr = y - yfar + far_field(h, x, round_s, round_vw)
        return np.max(np.linalg.norm(yr - y, axis=1) / np.linalg.norm(y, axis=1))

    def f32(a):
        return a.astype(np.float32).astype(np.float64)

    e32 = err(f32, f32)
    ebf = err(bf16_pair, f32)
    e1 = err(lambda a: bf16(a.astype(np.float32)).astype(np.float64), f32)
    assert e32 < 1e-6, e32                     # FP32 storage: far inside the 1e-5 budget
    assert 2.0 ** 4 * e32 < ebf < 1e-5, (e32, ebf)
    assert e1 > 1e-4 > 100 * ebf, (e1, ebf)    # one BF16 word would not do
