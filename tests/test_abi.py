"""CPU tests of the C-ABI library: it loads, exports every declared entry point, validates
arguments on the host, and its k-pair scheduler matches the oracle's definition exactly."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B


def test_library_exports_every_declared_symbol():
    declared = B.declared_symbols()
    assert len(declared) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    lib = B.lib()
    for s in declared:
        assert hasattr(lib, s)


def test_desc_layout_matches_header():
    # 16 int32 fields (mesh[3] counted as 3) then two doubles.
    assert ctypes.sizeof(B.dmet_emb_desc_t) == 16 * 4 + 16
    assert B.dmet_emb_desc_t.ortho_tol.offset == 64


def test_eri_bytes():
    d = dm.make_desc((2, 2, 1), 8, 40, 16)
    npair = 16 * 17 // 2
    assert dm.dmet_emb_eri_bytes(d, 0) == npair * (npair + 1) // 2 * 8
    assert dm.dmet_emb_eri_bytes(d, 1) == 0
    d = dm.make_desc((2, 2, 1), 8, 40, 16, sym=B.DMET_SYM_NONE)
    assert dm.dmet_emb_eri_bytes(d, 0) == 16 ** 4 * 16
    d = dm.make_desc((2, 2, 1), 8, 40, (5, 7), n_spin=2)
    pa, pb = 15, 28
    assert dm.dmet_emb_eri_bytes(d, 0) == pa * (pa + 1) // 2 * 8
    assert dm.dmet_emb_eri_bytes(d, 1) == pa * pb * 8
    assert dm.dmet_emb_eri_bytes(d, 2) == pb * (pb + 1) // 2 * 8
    d = dm.make_desc((2, 2, 1), 8, 40, (5, 7), n_spin=2, eri_pack=B.DMET_PACK_FULL)
    assert dm.dmet_emb_eri_bytes(d, 1) == 25 * 49 * 16
    d = dm.make_desc((2, 2, 1), 8, 40, (5, 7), n_spin=2, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_S4)
    from oracle import checks
    assert dm.dmet_emb_eri_bytes(d, 0) == checks.s4_size(5) * 16
    assert dm.dmet_emb_eri_bytes(d, 1) == 15 * 49 * 16
    assert dm.dmet_emb_eri_bytes(d, 2) == checks.s4_size(7) * 16


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1), (3, 2, 1), (2, 2, 2), (6, 6, 1),
                                  (4, 4, 4), (3, 3, 3), (5, 1, 2), (16, 16, 16)])
@pytest.mark.parametrize("sym", [0, 1])
def test_schedule_matches_oracle(mesh, sym):
    d = dm.make_desc(mesh, 2, 3, 1, sym=sym, eri_pack=B.DMET_PACK_FULL)
    got = dm.dmet_emb_schedule(d)
    if int(np.prod(mesh)) > 512:
        # Large mesh: invariants only (the oracle's pure-Python loops would be slow).
        nk = int(np.prod(mesh))
        assert int(got["q_weight"].sum()) == nk
        return
    ref = oracle.schedule(mesh, bool(sym))
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


BAD = {
    "mesh0": dict(mesh=(0, 1, 1)),
    "nk_too_big": dict(mesh=(17, 16, 16)),
    "n_ao": dict(n_ao=0),
    "n_aux": dict(n_aux=0),
    "n_spin": dict(n_spin=3),
    "n_emb0": dict(n_emb=0),
    "n_emb_big": dict(n_emb=4 * 8 + 1),
    "ck_norm": dict(ck_norm=2),
    "sym": dict(sym=5),
    "pack": dict(eri_pack=7),
    "s8_needs_real": dict(sym=0, eri_pack=1),
    "prec": dict(prec=9),
    "check_l": dict(check_l=3),
    "l_layout": dict(l_layout=2),
    "reduced_needs_real": dict(l_layout=1, sym=0),
    "reduced_needs_s8": dict(l_layout=1, eri_pack=2),
    "reduced_no_check_l": dict(l_layout=1, check_l=1),
    "shard_empty": dict(q_range=(2, 2)),
    "shard_reversed": dict(q_range=(3, 1)),
    "shard_past_mesh": dict(q_range=(0, 5)),
    "shard_negative": dict(q_range=(-1, 2)),
}


@pytest.mark.parametrize("name", sorted(BAD))
def test_invalid_descriptor_rejected_on_host(name):
    kw = dict(mesh=(2, 2, 1), n_ao=8, n_aux=40, n_emb=16)
    kw.update(BAD[name])
    d = dm.make_desc(**kw)
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(d)
    assert e.value.status == B.DMET_ERR_INVALID_ARG
    assert dm.dmet_emb_eri_bytes(d, 0) == 0


def _reduced_pairs_from_oracle(mesh, q_range=None):
    """The reduced layout's pair list written out from the oracle's schedule definition."""
    s = oracle.schedule(mesh, True)
    nk = int(np.prod(mesh))
    lo, hi = (0, nk) if q_range is None else q_range
    out = []
    for w in (1, 2):
        for q in range(nk):
            if s["q_weight"][q] != w or not lo <= q < hi:
                continue
            for r in range(s["n_rep"][q]):
                k1 = s["rep_k1"][q, r]
                out.append(k1 * nk + s["k2_of"][q, k1])
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1), (3, 3, 1), (2, 2, 2), (4, 4, 4),
                                  (6, 6, 1), (5, 1, 2)])
def test_reduced_pairs_match_schedule(mesh):
    d = dm.make_desc(mesh, 2, 3, 1)
    got = dm.dmet_emb_l_pairs(d)
    assert np.array_equal(got, _reduced_pairs_from_oracle(mesh))
    nk = int(np.prod(mesh))
    # every (k1, k2) block is one of the listed blocks up to Hermiticity and time reversal
    neg = oracle.schedule(mesh, True)["neg"]
    listed = set(got.tolist())
    for k1 in range(nk):
        for k2 in range(nk):
            images = {k1 * nk + k2, k2 * nk + k1, neg[k1] * nk + neg[k2], neg[k2] * nk + neg[k1]}
            assert images & listed, (k1, k2)


def test_reduced_pairs_of_shards_partition_the_list():
    mesh = (4, 4, 4)
    full = dm.dmet_emb_l_pairs(dm.make_desc(mesh, 2, 3, 1))
    parts = [dm.dmet_emb_l_pairs(dm.make_desc(mesh, 2, 3, 1, q_range=r)) for r in ((0, 9), (9, 30), (30, 64))]
    for r, p in zip(((0, 9), (9, 30), (30, 64)), parts):
        assert np.array_equal(p, _reduced_pairs_from_oracle(mesh, r))
    assert sorted(np.concatenate(parts).tolist()) == sorted(full.tolist())
    assert sum(len(p) for p in parts) == len(full)


def test_reduced_pairs_unsupported_for_complex_orbitals():
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_l_pairs(dm.make_desc((2, 2, 1), 2, 3, 1, sym=B.DMET_SYM_NONE))
    assert e.value.status == B.DMET_ERR_UNSUPPORTED


def test_null_arguments():
    lib = B.lib()
    assert lib.dmet_emb_plan(None, 1, None, 0, None) == B.DMET_ERR_INVALID_ARG
    assert lib.dmet_emb_eri(None, None, None, None) == B.DMET_ERR_INVALID_ARG
    assert lib.dmet_emb_transform_3idx(None, 0, None, None, 0, 0, None) == B.DMET_ERR_INVALID_ARG
    assert lib.dmet_emb_status(None, 0, None) == B.DMET_ERR_INVALID_ARG
    assert lib.dmet_emb_destroy(None) == B.DMET_OK
    assert b"NULL" in lib.dmet_emb_last_error() or lib.dmet_emb_last_error() == b""


def test_plan_without_gpu_reports_cuda_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(dm.make_desc((2, 2, 1), 8, 40, 16))
    assert e.value.status == B.DMET_ERR_CUDA


@pytest.mark.parametrize("fields", [
    dict(n_ao=1 << 20, n_aux=1 << 20, n_emb=(1 << 26, 0)),   # products that would wrap a 64-bit size
    dict(n_ao=4096, n_aux=65536, n_emb=(2047, 0)),          # within the bounds, far beyond the scratch
    dict(mesh=(65, 1, 1)),
    dict(check_l=2),
    dict(l_layout=1),
    dict(q_range=(0, 1)),
])
def test_noalloc_rejects_descriptors_before_touching_the_gpu(fields):
    """No CUDA call happens for these: the bounds and the scratch size are checked first."""
    kw = dict(mesh=(2, 2, 1), n_ao=8, n_aux=40, n_emb=16)
    kw.update({k: v for k, v in fields.items() if k != "n_emb"})
    d = dm.make_desc(**kw)
    if "n_emb" in fields:
        d.n_emb[:] = list(fields["n_emb"])
    buf = np.zeros(4)
    with pytest.raises(B.DmetError) as e:
        B.dmet_emb_eri_noalloc(d, buf, [buf], [buf])
    assert e.value.status in (B.DMET_ERR_INVALID_ARG, B.DMET_ERR_UNSUPPORTED, B.DMET_ERR_OOM)


def test_partial_shard_needs_s8():
    d = dm.make_desc((2, 2, 1), 8, 40, 16, sym=B.DMET_SYM_NONE, eri_pack=B.DMET_PACK_S4, q_range=(0, 1))
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(d)
    assert e.value.status == B.DMET_ERR_UNSUPPORTED


@pytest.mark.parametrize("pack", [B.DMET_PACK_FULL, B.DMET_PACK_S4, B.DMET_PACK_AUTO])
def test_tensor_core_precisions_take_complex_orbitals(pack):
    """General orbitals pass validation with a tensor-core precision (the plan then needs a GPU);
    real orbitals on a tensor-core precision still need the 8-fold packed output."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    d = dm.make_desc((2, 2, 1), 8, 40, 16, sym=B.DMET_SYM_NONE, eri_pack=pack, prec=B.DMET_PREC_BF16X3)
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(d)
    assert e.value.status == B.DMET_ERR_CUDA
    d = dm.make_desc((2, 2, 1), 8, 40, 16, eri_pack=B.DMET_PACK_FULL, prec=B.DMET_PREC_BF16X3)
    with pytest.raises(B.DmetError) as e:
        dm.dmet_emb_plan(d)
    assert e.value.status == B.DMET_ERR_UNSUPPORTED
