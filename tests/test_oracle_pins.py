"""Pins of the CPU oracle against facts that do not go through the oracle itself.

* P1 brute force: the real-space supercell transformation (no k-points) on tiny meshes.
* Golden: hand-derived worked examples (tests/golden/hand_supercell.json).
* P2 Nk = 1 reduces to the molecular density-fitted transform.
* P3/P4 permutational symmetry and vanishing imaginary parts for real orbitals.
* P5 the ERI supermatrix is a Gram matrix: Hermitian PSD of bounded rank.
* P6 invariance under a unitary rotation of the embedding orbitals.
* P7 impurity block of DMET-structured orbitals = the reference-cell AO ERI.
* P8 orthonormality of the generated orbitals.
* P9 exactness of orbital-column subsets.
* Planted mistakes: mutated copies of the oracle fail the pins.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import mesh as omesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_supercell.json")

MESHES = [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1), (2, 3, 1), (2, 2, 2)]


def small_spec(mesh, n_ao=3, n_aux=5, n_emb=4, seed=7, decay=0.6, **kw):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, 1, decay, 0.0, seed, "small", **kw)


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("mesh", MESHES)
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_brute_force_supercell(mesh, ck_norm):
    spec = small_spec(mesh, n_emb=min(5, 3 * int(np.prod(mesh))))
    B = synth.real_space_B(spec)
    csc = synth.supercell_orbitals(spec)
    L = synth.fourier_L(B, spec.mesh)
    C = synth.bloch_orbitals(csc, spec.mesh, ck_norm)
    eri = oracle.embedded_eri(L, C, spec.mesh, ck_norm=ck_norm)
    ref = oracle.supercell_eri(B, spec.mesh, csc)
    assert rel(eri, ref) < 1e-12
    assert np.abs(eri.imag).max() < 1e-12 * np.abs(ref).max()


def test_brute_force_complex_orbitals():
    spec = small_spec((3, 2, 1), n_emb=5)
    B = synth.real_space_B(spec)
    csc = synth.complex_supercell_orbitals(spec)
    L = synth.fourier_L(B, spec.mesh)
    eri = oracle.embedded_eri(L, synth.bloch_orbitals(csc, spec.mesh), spec.mesh)
    ref = oracle.supercell_eri(B, spec.mesh, csc)
    assert rel(eri, ref) < 1e-12
    assert np.abs(ref.imag).max() > 1e-3 * np.abs(ref).max()


def test_brute_force_unrestricted():
    spec = small_spec((2, 2, 1), n_emb=5)
    B = synth.real_space_B(spec)
    ca, cb = synth.supercell_orbitals(spec, 0), synth.supercell_orbitals(spec, 1)
    L = synth.fourier_L(B, spec.mesh)
    eri = oracle.embedded_eri(L, synth.bloch_orbitals(ca, spec.mesh), spec.mesh,
                              Cb=synth.bloch_orbitals(cb, spec.mesh))
    ref = oracle.supercell_eri(B, spec.mesh, ca, cb)
    assert rel(eri, ref) < 1e-12


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_hand_examples(case):
    mesh = tuple(case["mesh"])
    nk = int(np.prod(mesh))
    Bmat = np.array(case["B"], dtype=np.float64)
    B = Bmat.reshape(1, 1, nk, 1, nk)
    csc = np.eye(nk)
    L = synth.fourier_L(B, mesh)
    C = synth.bloch_orbitals(csc, mesh)
    eri = oracle.embedded_eri(L, C, mesh)
    brute = oracle.supercell_eri(B, mesh, csc)
    for (i, j, k, l), v in case["entries"]:
        assert abs(eri[i, j, k, l] - v) < 1e-12
        assert abs(brute[i, j, k, l] - v) < 1e-12
    if "packed_s8" in case:
        np.testing.assert_allclose(oracle.pack_s8(eri.real), case["packed_s8"], atol=1e-12)


def test_nk1_is_molecular_df():
    spec = small_spec((1, 1, 1), n_ao=6, n_aux=9, n_emb=5)
    L, (C,), _ = synth.make_problem(spec)
    eri = oracle.embedded_eri(L, C, spec.mesh)
    # Textbook molecular DF: (ij|kl) = sum_P (C^T L_P C)_ij (C^T L_P C)_kl.
    Lmo = np.einsum("mi,Pmn,nj->Pij", C[0].conj(), L[0, 0], C[0])
    ref = np.einsum("Pij,Pkl->ijkl", Lmo, Lmo)
    assert rel(eri, ref) < 1e-13


def _problem(mesh=(2, 3, 1), n_emb=6, real=True, seed=11):
    spec = small_spec(mesh, n_ao=3, n_aux=6, n_emb=n_emb, seed=seed)
    L, (C,), (csc,) = synth.make_problem(spec)
    if not real:
        # Complex real-space orbitals: orthonormal, not time-reversal symmetric.
        C = synth.bloch_orbitals(synth.complex_supercell_orbitals(spec), spec.mesh)
    return spec, L, C


@pytest.mark.parametrize("real", [True, False])
def test_permutational_symmetry(real):
    spec, L, C = _problem(real=real)
    eri = oracle.embedded_eri(L, C, spec.mesh)
    s = np.abs(eri).max()
    assert np.abs(eri - eri.transpose(2, 3, 0, 1)).max() < 1e-12 * s      # (ij|kl) = (kl|ij)
    assert np.abs(eri - eri.transpose(1, 0, 3, 2).conj()).max() < 1e-12 * s  # (ij|kl) = (ji|lk)*
    if real:
        assert np.abs(eri.imag).max() < 1e-12 * s
        assert np.abs(eri - eri.transpose(1, 0, 2, 3)).max() < 1e-12 * s
        assert np.abs(eri - eri.transpose(0, 1, 3, 2)).max() < 1e-12 * s
    else:
        assert np.abs(eri.imag).max() > 1e-6 * s
        assert oracle.orthonormality_error(C) < 1e-13


@pytest.mark.parametrize("real", [True, False])
def test_gram_psd_and_rank(real):
    spec, L, C = _problem(real=real)
    n = C.shape[2]
    eri = oracle.embedded_eri(L, C, spec.mesh)
    # G[(ij), (lk)] = (ij|kl) is a Gram matrix of the (q, P) factors.
    G = eri.transpose(0, 1, 3, 2).reshape(n * n, n * n)
    assert np.abs(G - G.conj().T).max() < 1e-12 * np.abs(G).max()
    w = np.linalg.eigvalsh(0.5 * (G + G.conj().T))
    assert w.min() > -1e-12 * w.max()
    rank = int((w > 1e-10 * w.max()).sum())
    assert rank <= spec.nk * spec.n_aux


def test_unitary_invariance():
    spec, L, C = _problem()
    n = C.shape[2]
    eri = oracle.embedded_eri(L, C, spec.mesh)
    rng = np.random.default_rng(3)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    CU = np.einsum("kmi,ia->kma", C, U)
    eriU = oracle.embedded_eri(L, CU, spec.mesh)
    assert abs(np.linalg.norm(eriU) - np.linalg.norm(eri)) < 1e-12 * np.linalg.norm(eri)
    # Two-electron energy with a Hermitian density matrix D, rotated as D -> U+ D U.
    h = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    D = h @ h.conj().T
    DU = U.conj().T @ D @ U

    def e2(e, d):
        return 0.5 * (np.einsum("ijkl,ji,lk->", e, d, d) - 0.5 * np.einsum("ijkl,jk,li->", e, d, d))

    assert abs(e2(eriU, DU) - e2(eri, D)) < 1e-11 * abs(e2(eri, D))


def test_dmet_structured_impurity_block():
    spec = small_spec((2, 2, 1), n_ao=3, n_aux=5, n_emb=5)
    B = synth.real_space_B(spec)
    csc = synth.dmet_structured_orbitals(spec, n_imp=3)
    L = synth.fourier_L(B, spec.mesh)
    C = synth.bloch_orbitals(csc, spec.mesh)
    eri = oracle.embedded_eri(L, C, spec.mesh)
    # Closed form: impurity AOs sit in cell 0, so X_{R0} = B[P, :, -R0, :, -R0].
    nk, n_imp = spec.nk, 3
    ref = np.zeros((n_imp,) * 4)
    for r0 in range(nk):
        m = omesh.k_neg(r0, spec.mesh)  # cell -R0 (cells and k-points share the index)
        x = B[:, :n_imp, m, :n_imp, m]
        ref += np.einsum("Pij,Pkl->ijkl", x, x)
    assert rel(eri[:n_imp, :n_imp, :n_imp, :n_imp], ref) < 1e-12


@pytest.mark.parametrize("ck_norm", [0, 1])
def test_orthonormality(ck_norm):
    spec = small_spec((2, 2, 1), n_emb=6)
    _, (C,), _ = synth.make_problem(spec, ck_norm=ck_norm, with_L=False)
    assert oracle.orthonormality_error(C, ck_norm) < 1e-13
    assert oracle.realness_error(C, spec.mesh) < 1e-13
    bad = C.copy()
    bad[1, 0, 0] += 1e-6
    assert oracle.orthonormality_error(bad, ck_norm) > 1e-8
    assert oracle.orthonormality_error(C, 1 - ck_norm) > 1e-3


def test_column_subset_exact():
    spec, L, C = _problem(n_emb=6)
    S = np.array([4, 1, 5])
    eri = oracle.embedded_eri(L, C, spec.mesh)
    sub = oracle.embedded_eri(L, C[:, :, S], spec.mesh)
    assert rel(sub, eri[np.ix_(S, S, S, S)]) < 1e-13


def test_entries_match_full():
    spec, L, C = _problem()
    Lq = oracle.embedded_3idx(L, C, spec.mesh)
    eri = oracle.embedded_eri(L, C, spec.mesh, Lq_a=Lq)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, C.shape[2], (50, 4))
    got = oracle.eri_entries(Lq, Lq, spec.mesh, idx)
    assert rel(got, eri[tuple(idx.T)]) < 1e-13


def test_pack_roundtrip():
    spec, L, C = _problem()
    eri = oracle.embedded_eri(L, C, spec.mesh).real
    n = C.shape[2]
    packed = oracle.pack_s8(eri)
    assert packed.size == (n * (n + 1) // 2) * (n * (n + 1) // 2 + 1) // 2
    assert np.abs(oracle.unpack_s8(packed, n) - eri).max() < 1e-14 * np.abs(eri).max()


def test_mesh_arithmetic():
    mesh = (2, 3, 4)
    nk = 24
    for k in range(nk):
        assert omesh.k_index(omesh.k_triplet(k, mesh), mesh) == k
        assert omesh.k_add(k, omesh.k_neg(k, mesh), mesh) == 0
    assert omesh.k_triplet(23, mesh) == (1, 2, 3)
    assert omesh.k_add(omesh.k_index((1, 2, 3), mesh), omesh.k_index((1, 2, 2), mesh), mesh) == \
        omesh.k_index((0, 1, 1), mesh)


# ---------------------------------------------------------------------------------------------
# Planted mistakes: each mutation of the oracle's source must fail a pin.

MUTATIONS = {
    "no_conj_on_bra": ("C[k1].conj().T", "C[k1].T"),
    "second_factor_same_q": ("Lq_b[k_neg(q, mesh)]", "Lq_b[q]"),
    "dropped_ft_scale": ("scale = 1.0 / nk if ck_norm == 0 else 1.0", "scale = 1.0"),
    "dropped_contraction_scale": ("axes=([0], [0])) / nk", "axes=([0], [0]))"),
    "transposed_L": ("np.matmul(L[k1, k2], C[k2])", "np.matmul(L[k1, k2].transpose(0, 2, 1), C[k2])"),
    "swapped_k_of_L": ("np.matmul(L[k1, k2], C[k2])", "np.matmul(L[k2, k1], C[k2])"),
    "wrong_k_on_ket": ("np.matmul(L[k1, k2], C[k2])", "np.matmul(L[k1, k2], C[k1])"),
    "k2_minus_q": ("k2 = k_add(k1, q, mesh)", "k2 = k_add(k1, k_neg(q, mesh), mesh) if q % 2 else k_add(k1, q, mesh)"),
}


def _mutated_alg1(old, new):
    path = os.path.join(os.path.dirname(oracle.__file__), "alg1.py")
    with open(path) as f:
        src = f.read()
    assert src.count(old) >= 1, old
    ns = {"__name__": "oracle.alg1_mutant", "__package__": "oracle"}
    exec(compile(src.replace(old, new), "alg1_mutant", "exec"), ns)
    return ns


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name):
    ns = _mutated_alg1(*MUTATIONS[name])
    spec = small_spec((2, 3, 1), n_ao=3, n_aux=4, n_emb=5, seed=5)
    B = synth.real_space_B(spec)
    csc = synth.supercell_orbitals(spec)
    L = synth.fourier_L(B, spec.mesh)
    C = synth.bloch_orbitals(csc, spec.mesh)
    ref = oracle.supercell_eri(B, spec.mesh, csc)
    eri = ns["embedded_eri"](L, C, spec.mesh)
    assert rel(eri, ref) > 1e-6, name
    # The unmutated oracle passes the same pin.
    assert rel(oracle.embedded_eri(L, C, spec.mesh), ref) < 1e-12


# ---------------------------------------------------------------------------------------------
# Algorithm 1 with L streamed in blocks of aux functions (used for the full-size checks).

def _blocks(L, pb):
    return (L[:, :, p0:p0 + pb] for p0 in range(0, L.shape[2], pb))


@pytest.mark.parametrize("mesh", [(2, 2, 1), (3, 1, 1), (2, 3, 1)])
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_pblocks_brute_force_unrestricted(mesh, ck_norm):
    spec = small_spec(mesh, n_ao=3, n_aux=7, n_emb=5)
    B = synth.real_space_B(spec)
    ca, cb = synth.supercell_orbitals(spec, 0), synth.supercell_orbitals(spec, 1)
    L = synth.fourier_L(B, spec.mesh)
    Cs = [synth.bloch_orbitals(c, spec.mesh, ck_norm) for c in (ca, cb)]
    got = oracle.embedded_eri_pblocks(_blocks(L, 3), Cs, spec.mesh, ck_norm=ck_norm)
    assert sorted(got) == [(0, 0), (0, 1), (1, 1)]
    assert rel(got[(0, 0)], oracle.supercell_eri(B, spec.mesh, ca)) < 1e-12
    assert rel(got[(0, 1)], oracle.supercell_eri(B, spec.mesh, ca, cb)) < 1e-12
    assert rel(got[(1, 1)], oracle.supercell_eri(B, spec.mesh, cb)) < 1e-12


def test_pblocks_complex_orbitals():
    spec = small_spec((3, 2, 1), n_ao=2, n_aux=5, n_emb=4)
    B = synth.real_space_B(spec)
    csc = synth.complex_supercell_orbitals(spec)
    L = synth.fourier_L(B, spec.mesh)
    got = oracle.embedded_eri_pblocks(_blocks(L, 2), [synth.bloch_orbitals(csc, spec.mesh)], spec.mesh)
    assert rel(got[(0, 0)], oracle.supercell_eri(B, spec.mesh, csc)) < 1e-12


BLOCK_MUTATIONS = {
    "no_conj_on_bra": ("pair = C[k1].conj().T @", "pair = C[k1].T @"),
    "bra_rows_not_restacked": ("right.transpose(1, 0, 2).reshape(na, pb * n)", "right.reshape(na, pb * n)"),
    "result_not_untransposed": ("pair.reshape(n, pb, n).transpose(1, 0, 2)", "pair.reshape(pb, n, n)"),
    "second_factor_same_q": ("lq[b][k_neg(q, mesh)]", "lq[b][q]"),
    "ket_with_k1": ("@ C[k2]).reshape(pb, na, n)", "@ C[k1]).reshape(pb, na, n)"),
}


@pytest.mark.parametrize("name", sorted(BLOCK_MUTATIONS))
def test_planted_mistake_in_block_form_fails(name):
    ns = _mutated_alg1(*BLOCK_MUTATIONS[name])
    spec = small_spec((2, 3, 1), n_ao=3, n_aux=4, n_emb=5, seed=5)
    B = synth.real_space_B(spec)
    csc = synth.supercell_orbitals(spec)
    L = synth.fourier_L(B, spec.mesh)
    C = synth.bloch_orbitals(csc, spec.mesh)
    ref = oracle.supercell_eri(B, spec.mesh, csc)
    eri = ns["embedded_eri_pblocks"](_blocks(L, 3), [C], spec.mesh)[(0, 0)]
    assert rel(eri, ref) > 1e-6, name
    assert rel(oracle.embedded_eri_pblocks(_blocks(L, 3), [C], spec.mesh)[(0, 0)], ref) < 1e-12


# ---------------------------------------------------------------------------------------------
# 4-fold packing of a complex ERI: the layout's definition fixed by a table worked out by hand for two
# orbitals (pairs 00 -> 0, 10 -> 1, 11 -> 2; block A at IJ(IJ+1)/2 + KL; block B after the 6 entries of
# A, its only entry (10|01)); (position, stored as the conjugate?).
S4_HAND_N2 = {
    (0, 0, 0, 0): (0, False), (0, 0, 0, 1): (1, True), (0, 0, 1, 0): (1, False), (0, 0, 1, 1): (3, False),
    (0, 1, 0, 0): (1, True), (0, 1, 0, 1): (2, True), (0, 1, 1, 0): (6, False), (0, 1, 1, 1): (4, True),
    (1, 0, 0, 0): (1, False), (1, 0, 0, 1): (6, False), (1, 0, 1, 0): (2, False), (1, 0, 1, 1): (4, False),
    (1, 1, 0, 0): (3, False), (1, 1, 0, 1): (4, True), (1, 1, 1, 0): (4, False), (1, 1, 1, 1): (5, False),
}


def test_s4_layout_hand_table():
    from oracle import checks
    assert checks.s4_size(2) == 7
    for idx, want in S4_HAND_N2.items():
        assert checks._s4_home(*idx, 2) == want, idx


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_s4_every_slot_holds_one_orbit(n):
    """Each packed slot is the home of the 1, 2 or 4 entries of one symmetry orbit, and of nothing else."""
    from oracle import checks
    members = {}
    for idx in np.ndindex(n, n, n, n):
        p, c = checks._s4_home(*idx, n)
        members.setdefault(p, []).append((idx, c))
    assert sorted(members) == list(range(checks.s4_size(n)))
    for p, m in members.items():
        i, j, k, l = m[0][0]
        orbit = {(i, j, k, l), (k, l, i, j), (j, i, l, k), (l, k, j, i)}
        assert {x for x, _ in m} == orbit, (p, m)
        # the swap keeps the conjugation flag, the pair transposition flips it
        flags = dict(m)
        assert flags[(i, j, k, l)] == flags[(k, l, i, j)] != flags[(j, i, l, k)] or (i, j, k, l) == (j, i, l, k) \
            or (i, j, k, l) == (l, k, j, i)


@pytest.mark.parametrize("mesh,n,complex_orbitals", [((3, 2, 1), 4, True), ((2, 2, 1), 5, True), ((3, 1, 1), 3, False)])
def test_s4_roundtrip_of_the_oracle_eri(mesh, n, complex_orbitals):
    from oracle import checks
    spec = small_spec(mesh, n_ao=3, n_aux=5, n_emb=n)
    L = synth.make_L(spec)
    csc = synth.complex_supercell_orbitals(spec) if complex_orbitals else synth.supercell_orbitals(spec)
    eri = oracle.embedded_eri(L, synth.bloch_orbitals(csc, mesh), mesh)
    packed = checks.pack_s4(eri)
    assert len(packed) == checks.s4_size(n)
    assert rel(checks.unpack_s4(packed, n), eri) < 1e-13
    if complex_orbitals:
        assert np.abs(packed.imag).max() > 1e-3 * np.abs(packed).max()
