"""GPU parity of the split-BF16 (tcgen05) path against the FP64 CPU oracle, through the C ABI.

Tolerance: 1e-6 relative Frobenius norm for the mixed path (three bf16 slices carry ~24
bits per operand; FP32 accumulation per short K segment; sums across segments in an exact
two-float representation), and the maximum error relative to max |(ij|kl)| below 1e-6 too.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, run_eri, s8_index, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def spec_of(mesh, n_ao, n_aux, n_emb, n_spin=1, seed=21, decay=0.6, c_log_range=0.0):
    return synth.LatticeSpec(tuple(mesh), n_ao, n_aux, n_emb, n_spin, decay, c_log_range, seed, "m")


def desc_of(spec, n_emb=None, **kw):
    ne = n_emb or ([spec.n_emb, spec.n_emb] if spec.n_spin == 2 else [spec.n_emb, 0])
    return B.make_desc(spec.mesh, spec.n_ao, spec.n_aux, ne, n_spin=spec.n_spin, prec=B.DMET_PREC_BF16X3, **kw)


def check(got, ref):
    assert got.shape == ref.shape
    assert np.isfinite(got).all()
    e = rel_fro(got, ref)
    m = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < TOL and m < TOL, (e, m)
    return e


CASES = [
    ((2, 2, 1), 8, 40, 16),
    ((1, 1, 1), 5, 7, 3),
    ((3, 1, 1), 5, 7, 1),
    ((2, 3, 1), 6, 11, 33),
    ((3, 3, 1), 10, 37, 70),
    ((2, 2, 2), 4, 9, 20),
    ((3, 2, 1), 24, 60, 130),   # more than one 128-row tile of pairs and of (P, j) rows
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + f"_ao{c[1]}_aux{c[2]}_n{c[3]}")
@pytest.mark.parametrize("ck_norm", [0, 1])
def test_mixed_eri_matches_oracle(torch, case, ck_norm):
    mesh, nao, naux, n = case
    spec = spec_of(mesh, nao, naux, n)
    L, Cs, _ = synth.make_problem(spec, ck_norm=ck_norm)
    (got,), st, stats = run_eri(torch, desc_of(spec, ck_norm=ck_norm), L, Cs)
    assert st == B.DMET_OK, (st, stats)
    check(got, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh, ck_norm=ck_norm).real))


def test_mixed_unrestricted_blocks(torch):
    spec = spec_of((2, 2, 1), 5, 9, 6, n_spin=2)
    L = synth.make_L(spec)
    ca = synth.bloch_orbitals(synth.supercell_orbitals(spec, 0), spec.mesh)
    cb = synth.bloch_orbitals(synth.supercell_orbitals(synth.spec_with(spec, n_emb=9), 1), spec.mesh)
    (aa, ab, bb), st, _ = run_eri(torch, desc_of(spec, n_emb=[6, 9]), L, [ca, cb])
    assert st == B.DMET_OK
    check(aa, oracle.pack_s8(oracle.embedded_eri(L, ca, spec.mesh).real))
    check(bb, oracle.pack_s8(oracle.embedded_eri(L, cb, spec.mesh).real))
    check(ab, oracle.pair_matrix(oracle.embedded_eri(L, ca, spec.mesh, Cb=cb).real).ravel())


def test_mixed_log_uniform_orbitals(torch):
    """Orbital entries spread over four decades (the silicon-shaped precision study's recipe)."""
    spec = spec_of((2, 2, 2), 6, 15, 24, c_log_range=4.0)
    L, Cs, _ = synth.make_problem(spec)
    (got,), st, _ = run_eri(torch, desc_of(spec), L, Cs)
    assert st == B.DMET_OK
    check(got, oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real))


def test_mixed_small_workspace_same_result(torch):
    spec = spec_of((3, 3, 1), 5, 12, 11)
    L, Cs, _ = synth.make_problem(spec)
    (a,), _, _ = run_eri(torch, desc_of(spec), L, Cs)
    (b,), _, _ = run_eri(torch, desc_of(spec), L, Cs, workspace_limit=16 << 20)
    assert rel_fro(b, a) < 1e-7


def test_mixed_hbn_full_size_sampled(torch):
    """h-BN-shaped 6x6x1 workload at full size; every entry on a seeded 16-orbital subset."""
    spec = synth.CONFIGS["hbn_6x6x1"]
    L, (C,), _ = synth.make_problem(spec)
    (got,), st, stats = run_eri(torch, desc_of(spec), L, [C])
    assert st == B.DMET_OK, stats
    rng = np.random.default_rng(0)
    S = np.sort(rng.choice(spec.n_emb, 16, replace=False))
    Lq = oracle.embedded_3idx(L, C[:, :, S], spec.mesh)
    i, j, k, l = np.meshgrid(*([np.arange(16)] * 4), indexing="ij")
    idx = np.stack([i.ravel(), j.ravel(), k.ravel(), l.ravel()], 1)
    ref = oracle.eri_entries(Lq, Lq, spec.mesh, idx).real
    check(got[s8_index(*(S[idx.T]))], ref)


@pytest.mark.parametrize("bn", [128, 112, 96])
def test_mixed_tile_widths(torch, bn, tmp_path, monkeypatch):
    """Every output tile width of the transform GEMMs gives the same parity (forced through the
    tuning cache that dmet_emb_plan reads)."""
    import paper_1909_08596_gb300 as dm
    spec = spec_of((3, 2, 1), 10, 30, 55)
    L, Cs, _ = synth.make_problem(spec)
    cache = tmp_path / "tune.txt"
    cache.write_text(f"3 2 1 10 30 55 0 1 {bn} {bn}\n")
    monkeypatch.setenv("DMET_TUNE_CACHE", str(cache))
    d = desc_of(spec)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    out = torch.empty(B.dmet_emb_eri_bytes(d, 0) // 8, dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        assert dm.dmet_emb_tile_widths(plan, 0) == [bn, bn]
        dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    check(out.cpu().numpy(), oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real))


def test_mixed_autotune(torch, tmp_path, monkeypatch):
    import paper_1909_08596_gb300 as dm
    spec = spec_of((3, 3, 1), 10, 37, 70)
    L, Cs, _ = synth.make_problem(spec)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("DMET_TUNE_CACHE", str(cache))
    d = desc_of(spec)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    out = torch.empty(B.dmet_emb_eri_bytes(d, 0) // 8, dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_autotune(plan, [Ld], [Cd], [[out]])
        widths = dm.dmet_emb_tile_widths(plan, 0)
        parts = dm.dmet_emb_split_parts(plan, 0)
        out.fill_(float("nan"))
        dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    assert widths[0] in (128, 112, 96) and widths[1] in (128, 112, 96)
    fields = cache.read_text().split()
    assert fields[-3:-1] == [str(widths[0]), str(widths[1])]
    assert int(fields[-1]) in (0, 1, 2, 4, 8)
    assert parts[0][1] >= 1
    check(out.cpu().numpy(), oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real))


@pytest.mark.parametrize("check_l", [0, 1])
def test_mixed_host_inputs_match_device(torch, check_l):
    """Host-resident L and C give the device result: only the (k1, k2) blocks the schedule reads
    are transferred (all of them with check_l), and nothing else of L is needed."""
    spec = spec_of((3, 3, 1), 6, 11, 20)
    L, Cs, _ = synth.make_problem(spec)
    d = desc_of(spec, check_l=check_l)
    dev, st1, _ = run_eri(torch, d, L, Cs)
    host, st2, _ = run_eri(torch, d, L, Cs, host=True)
    assert st1 == st2 == B.DMET_OK
    assert np.array_equal(dev[0], host[0])
    check(host[0], oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real))


def test_mixed_pinned_host_inputs_match_device(torch):
    """Pinned host L (which the GPU can address directly) gives the device result."""
    import paper_1909_08596_gb300 as dm
    spec = spec_of((3, 3, 1), 6, 11, 20)
    L, Cs, _ = synth.make_problem(spec)
    d = desc_of(spec)
    dev, st1, _ = run_eri(torch, d, L, Cs)
    Lh = torch.from_numpy(L).pin_memory()
    Ch = [torch.from_numpy(c).pin_memory() for c in Cs]
    Oh = [torch.empty(dm.dmet_emb_eri_bytes(d, 0) // 8, dtype=torch.float64).pin_memory()]
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        for _ in range(2):  # the second call reuses the staging buffer
            dm.dmet_emb_eri(plan, [Lh], [Ch], [Oh])
            torch.cuda.synchronize()
            st2, _ = dm.dmet_emb_status(plan, 0)
            assert st1 == st2 == B.DMET_OK
            assert np.array_equal(dev[0], Oh[0].numpy())
    finally:
        dm.dmet_emb_destroy(plan)


@pytest.mark.parametrize("qblock", [1, 3])
def test_mixed_qblock_cap_matches_oracle(torch, monkeypatch, qblock):
    """A plan built under DMET_QBLOCK (smaller q-blocks, more of them) gives the oracle's ERI from
    device and from host inputs alike; the host inputs then stream in many pitched copies."""
    spec = spec_of((4, 3, 1), 6, 11, 20)
    L, Cs, _ = synth.make_problem(spec)
    d = desc_of(spec)
    ref = oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real)
    base, st0, _ = run_eri(torch, d, L, Cs)
    monkeypatch.setenv("DMET_QBLOCK", str(qblock))
    dev, st1, _ = run_eri(torch, d, L, Cs)
    host, st2, _ = run_eri(torch, d, L, Cs, host=True)
    assert st0 == st1 == st2 == B.DMET_OK
    assert np.array_equal(dev[0], host[0])
    check(dev[0], ref)
    assert rel_fro(dev[0], base[0]) < TOL


@pytest.mark.parametrize("split", [1, 2, 8])
def test_mixed_split_parts(torch, split, tmp_path, monkeypatch):
    """The K split of the contraction's last wave (forced through the tuning cache) changes only
    the summation grouping of the tail tiles: parity holds for every factor."""
    import paper_1909_08596_gb300 as dm
    spec = spec_of((3, 3, 1), 10, 37, 70)
    L, Cs, _ = synth.make_problem(spec)
    cache = tmp_path / "tune.txt"
    cache.write_text(f"3 3 1 10 37 70 0 1 128 128 {split}\n")
    monkeypatch.setenv("DMET_TUNE_CACHE", str(cache))
    d = desc_of(spec)
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    out = torch.full((B.dmet_emb_eri_bytes(d, 0) // 8,), float("nan"), dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(d, stream=torch.cuda.current_stream().cuda_stream)
    try:
        tiles, f = dm.dmet_emb_split_parts(plan, 0)[0]
        dm.dmet_emb_eri(plan, [Ld], [Cd], [[out]])
        st, _ = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    assert st == B.DMET_OK
    assert f == (1 if split == 1 or tiles == 0 else split) or (tiles > 0 and f < split)
    check(out.cpu().numpy(), oracle.pack_s8(oracle.embedded_eri(L, Cs[0], spec.mesh).real))


def test_job_pacing_changes_no_result(torch, monkeypatch):
    """The contraction's job pacing (DMET_TC_PACE, on by default) only orders when the CTAs load their
    tiles: the results are bit-for-bit those of the unpaced launch."""
    spec = spec_of((3, 3, 1), 10, 37, 70)
    L, Cs, _ = synth.make_problem(spec)
    d = desc_of(spec)
    monkeypatch.setenv("DMET_TC_PACE", "0")
    a, st1, _ = run_eri(torch, d, L, Cs)
    monkeypatch.setenv("DMET_TC_PACE", "1")
    b, st2, _ = run_eri(torch, d, L, Cs)
    assert st1 == st2 == B.DMET_OK
    assert np.array_equal(a[0], b[0])
