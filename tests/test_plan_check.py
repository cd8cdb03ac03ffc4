"""Host-only checks of the execution plan through h2_plan_check (no GPU).

The library builds the cluster tree, the block partition, the product's
passes and the dataflow ticket orders on the host exactly as h2_assemble does
and checks the invariants its kernels rely on (legal bulk copies, a
topological ticket order, consistent expected signal counts).  The tree and
the block partition are also compared with the oracle's own implementation of
the same rules.
"""
import itertools

import numpy as np
import pytest

import oracle
import paper_1811_05731_gb300 as pkg
import synth

MESHES = {
    "ico3": lambda: synth.icosphere(3),
    "cube12": lambda: synth.cube_surface(12),
    "cube_sphere9": lambda: synth.cube_sphere(9),
    "film_small": lambda: synth.film_box(40, 2, 1000.0, 10.0),
    "ellipsoid4": lambda: synth.ellipsoid(4),
    "torus": lambda: synth.torus_surface(48, 24),
    "prism": lambda: synth.box_surface(20, 40, 2, 10.0, 20.0, 1.0),
}


@pytest.fixture(scope="module")
def L():
    pkg.build()
    return pkg.load()


@pytest.mark.parametrize("name", sorted(MESHES))
def test_plans_are_sound_for_every_form(L, name):
    mesh = MESHES[name]()
    for (m, leaf), prec, r, workers in itertools.product(((3, 16), (4, 32), (5, 64)), (0, 1, 2, 3),
                                                         (1, 3, 16, 32), (1, 456)):
        rep = pkg.h2_plan_check(mesh.xyz, mesh.tri, workers, m=m, leaf=leaf, precision=prec, max_rhs=r)
        assert rep["violations"] == 0, (name, m, leaf, prec, r, workers, rep)
        assert rep["n_regions"] == 3 * rep["n_clusters"]
        # without admissible blocks the split order (everything but the near
        # field) is empty
        assert rep["makespan_us"] > 0.0 and rep["n_segments"] > rep["n_split_segments"] >= 0
        assert (rep["n_split_segments"] == 0) == (rep["n_far_blocks"] == 0)


def test_evaluated_coupling_plans_are_sound(L):
    mesh = synth.cube_sphere(9)
    for r in (1, 16):
        rep = pkg.h2_plan_check(mesh.xyz, mesh.tri, 456, m=4, leaf=20, precision=pkg.FP32, max_rhs=r,
                                coupling=pkg.COUPLING_ON_THE_FLY)
        assert rep["violations"] == 0, rep


@pytest.mark.parametrize("name", ["ico3", "cube12", "ellipsoid4", "torus", "prism"])
def test_tree_and_blocks_match_the_oracle(L, name):
    mesh = MESHES[name]()
    for m, leaf, eta in ((3, 16, 2.0), (4, 32, 1.0), (4, 64, 2.0)):
        rep = pkg.h2_plan_check(mesh.xyz, mesh.tri, 456, m=m, leaf=leaf, eta=eta)
        h = oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, eta, store=False)
        assert (rep["n_clusters"], rep["n_levels"], rep["n_far_blocks"], rep["n_near_blocks"]) == \
            (h.n_clusters, h.n_levels, h.n_far, h.n_near), (name, m, leaf, eta)


def test_plan_bytes_cover_the_stored_coefficients(L):
    """FP64 plan: every near entry and coupling coefficient of the oracle's
    operator is streamed once per product, and at most every leaf basis of
    both sides and every transfer of both passes besides (clusters outside
    all admissible blocks need none), with a few per cent of 16-byte padding."""
    mesh = synth.cube_surface(12)
    m, leaf = 4, 32
    rep = pkg.h2_plan_check(mesh.xyz, mesh.tri, 456, m=m, leaf=leaf)
    h = oracle.H2Oracle(mesh.xyz, mesh.tri, m, leaf, 2.0, store=False)
    t = h.tree()
    k = h.k
    leaves = t["child0"] < 0
    lower = h.near_entries + h.n_far * k * k
    upper = lower + 2 * int(np.sum(t["size"][leaves])) * k + 2 * (h.n_clusters - 1) * k * k
    assert 8 * lower < rep["bytes_streamed"] <= 1.05 * 8 * upper, (rep["bytes_streamed"], 8 * lower, 8 * upper)


def test_invalid_meshes_and_parameters_are_refused(L):
    mesh = synth.icosphere(2)
    with pytest.raises(pkg.H2Error):
        pkg.h2_plan_check(mesh.xyz, mesh.tri[1:])                 # open
    with pytest.raises(pkg.H2Error):
        pkg.h2_plan_check(mesh.xyz, mesh.tri[:, ::-1])            # inward
    with pytest.raises(pkg.H2Error):
        pkg.h2_plan_check(mesh.xyz, mesh.tri, m=9)
    with pytest.raises(pkg.H2Error):
        pkg.h2_plan_check(mesh.xyz, mesh.tri, 0)
    with pytest.raises(pkg.H2Error):
        pkg.h2_plan_check(mesh.xyz, mesh.tri, schedule=7)
