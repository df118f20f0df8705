"""Helpers for the GPU tests: run the library through its C ABI on torch-owned buffers."""
import numpy as np

import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU test needs CUDA")
    from paper_1909_08596_gb300 import build
    build.build()
    return torch


def rel_fro(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def s8_index(i, j, k, l):
    i, j, k, l = map(np.asarray, (i, j, k, l))
    I, J = np.maximum(i, j), np.minimum(i, j)
    K, Lx = np.maximum(k, l), np.minimum(k, l)
    ij = I * (I + 1) // 2 + J
    kl = K * (K + 1) // 2 + Lx
    P, Q = np.maximum(ij, kl), np.minimum(ij, kl)
    return P * (P + 1) // 2 + Q


def ab_index(i, j, k, l, nb):
    i, j, k, l = map(np.asarray, (i, j, k, l))
    I, J = np.maximum(i, j), np.minimum(i, j)
    K, Lx = np.maximum(k, l), np.minimum(k, l)
    npb = nb * (nb + 1) // 2
    return (I * (I + 1) // 2 + J) * npb + (K * (K + 1) // 2 + Lx)


def out_buffers(torch, desc, device="cuda"):
    nblk = 1 if desc.n_spin == 1 else 3
    full = desc.eri_pack == B.DMET_PACK_FULL or (desc.eri_pack == B.DMET_PACK_AUTO and desc.sym == B.DMET_SYM_NONE)
    outs = []
    for b in range(nblk):
        nbytes = dm.dmet_emb_eri_bytes(desc, b)
        if full:
            outs.append(torch.empty(nbytes // 16, dtype=torch.complex128, device=device))
        else:
            outs.append(torch.empty(nbytes // 8, dtype=torch.float64, device=device))
    return outs


def run_eri(torch, desc, L, Cs, host=False, workspace_limit=0):
    """Returns (list of numpy output blocks, status, stats)."""
    if host:
        Ld = np.ascontiguousarray(L)
        Cd = [np.ascontiguousarray(c) for c in Cs]
        outs = [np.empty(dm.dmet_emb_eri_bytes(desc, b) // 8, dtype=np.float64)
                for b in range(1 if desc.n_spin == 1 else 3)]
        full = desc.eri_pack == B.DMET_PACK_FULL or (desc.eri_pack == 0 and desc.sym == 0)
        if full:
            outs = [o.view(np.complex128) for o in outs]
    else:
        Ld = torch.from_numpy(L).cuda()
        Cd = [torch.from_numpy(c).cuda() for c in Cs]
        outs = out_buffers(torch, desc)
    plan = dm.dmet_emb_plan(desc, stream=torch.cuda.current_stream().cuda_stream, workspace_limit=workspace_limit)
    try:
        dm.dmet_emb_eri(plan, [Ld], [Cd], [outs])
        st, stats = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    res = [o if isinstance(o, np.ndarray) else o.cpu().numpy() for o in outs]
    return res, st, stats


def run_3idx(torch, desc, L, Cs, q_begin, q_end):
    Ld = torch.from_numpy(L).cuda()
    Cd = [torch.from_numpy(c).cuda() for c in Cs]
    ns = [desc.n_emb[s] for s in range(desc.n_spin)]
    outs = [torch.empty((q_end - q_begin, desc.n_aux, n, n), dtype=torch.complex128, device="cuda") for n in ns]
    plan = dm.dmet_emb_plan(desc, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_transform_3idx(plan, 0, Ld, Cd, q_begin, q_end, outs)
        st, stats = dm.dmet_emb_status(plan, 0)
    finally:
        dm.dmet_emb_destroy(plan)
    return [o.cpu().numpy() for o in outs], st, stats
