"""Pins of the oracle's k-pair schedule (section 2.1, Algorithm 1 loops) by invariants and by
reconstructing the oracle's own L^q and ERI from the reduced pair set."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mesh as omesh

MESHES = [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2), (6, 6, 1), (4, 4, 4), (3, 3, 3), (5, 1, 2)]


@pytest.mark.parametrize("mesh", MESHES)
@pytest.mark.parametrize("real", [False, True])
def test_schedule_invariants(mesh, real):
    s = oracle.schedule(mesh, real)
    nk = int(np.prod(mesh))
    for q in range(nk):
        tq = omesh.k_triplet(q, mesh)
        for k1 in range(nk):
            a, b = omesh.k_triplet(k1, mesh), omesh.k_triplet(int(s["k2_of"][q, k1]), mesh)
            assert all((b[d] - a[d] - tq[d]) % mesh[d] == 0 for d in range(3))
        covered = []
        for r in range(s["n_rep"][q]):
            k1 = int(s["rep_k1"][q, r])
            partner = omesh.k_neg(omesh.k_add(k1, q, mesh), mesh)
            covered += [k1] if (s["rep_half"][q, r] or not real) else [k1, partner]
            if s["rep_half"][q, r]:
                t = omesh.k_triplet(k1, mesh)
                assert all((2 * t[d] + tq[d]) % mesh[d] == 0 for d in range(3))
        assert sorted(covered) == list(range(nk))
    assert int(s["q_weight"].sum()) == nk
    if real:
        for q in range(nk):
            if s["q_weight"][q]:
                assert s["q_weight"][q] == (1 if omesh.k_neg(q, mesh) == q else 2)


@pytest.mark.parametrize("mesh", [(2, 3, 1), (3, 3, 1), (2, 2, 2)])
def test_reduced_pairs_rebuild_the_oracle(mesh):
    spec = synth.LatticeSpec(mesh, 3, 4, 5, 1, 0.6, 0.0, 13, "s")
    L, (C,), _ = synth.make_problem(spec)
    nk = spec.nk
    s = oracle.schedule(mesh, True)
    Lq = oracle.embedded_3idx(L, C, mesh)
    eri = oracle.embedded_eri(L, C, mesh, Lq_a=Lq)
    rebuilt = np.zeros_like(Lq)
    for q in range(nk):
        Z = 0
        for r in range(s["n_rep"][q]):
            k1 = int(s["rep_k1"][q, r])
            k2 = int(s["k2_of"][q, k1])
            y = np.matmul(C[k1].conj().T[None], np.matmul(L[k1, k2], C[k2]))
            Z = Z + (0.5 if s["rep_half"][q, r] else 1.0) * y
        rebuilt[q] = (Z + Z.transpose(0, 2, 1)) / nk
    assert np.abs(rebuilt - Lq).max() < 1e-13 * np.abs(Lq).max()
    # Contraction over q <= -q with the weights, real parts only.
    n = C.shape[2]
    acc = np.zeros((n, n, n, n))
    for q in range(nk):
        w = s["q_weight"][q]
        if w:
            a = Lq[q]
            acc += w * (np.einsum("Pij,Pkl->ijkl", a.real, a.real) + np.einsum("Pij,Pkl->ijkl", a.imag, a.imag)) / nk
    assert np.abs(acc - eri.real).max() < 1e-13 * np.abs(eri).max()


def test_pair_blocks_of_the_reduced_layout_match_full_L():
    """The generator's per-pair L blocks (for a reduced input layout) equal the full L's blocks, for the
    pairs the 8-fold schedule reads, generated P-block by P-block."""
    import synth
    spec = synth.spec_with(synth.CONFIGS["tiny_2x2x1"], mesh=(3, 2, 1), n_ao=3, n_aux=7)
    from oracle.schedule import schedule
    s = schedule(spec.mesh, real=True)
    nk = spec.nk
    pairs = sorted({int(k1) * nk + int(s["k2_of"][q][k1]) for q in range(nk) if s["q_weight"][q] > 0
                    for k1 in s["rep_k1"][q][:s["n_rep"][q]]})
    full = synth.make_L(spec)
    red = synth.make_L_pairs(spec, pairs, p_block=3)
    for e, p in enumerate(pairs):
        np.testing.assert_array_equal(red[e], full[p // nk, p % nk])
    assert len(pairs) < nk * nk / 2
