"""A bounded device wait that expires is reported, not hung on: with the test hook that makes the
tensor-core kernels' producer withhold its copies, the MMA thread's and the epilogue's waits on
mbarriers that nobody arrives at expire after the plan's wait limit (a few milliseconds here), with no
copy and no MMA in flight; dmet_emb_status returns DMET_ERR_TIMEOUT through the device error word, and
the same plan then runs normally (the context stays usable)."""
import numpy as np
import pytest

import oracle
import synth
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

from gpu_helpers import rel_fro, torch_cuda

pytestmark = pytest.mark.gpu


def test_expired_wait_returns_timeout_and_plan_recovers():
    torch = torch_cuda()
    spec = synth.CONFIGS["tiny_2x2x1"]
    L, (C,), _ = synth.make_problem(spec)
    desc = dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb, prec=B.DMET_PREC_BF16X3)
    Ld, Cd = torch.from_numpy(L).cuda(), torch.from_numpy(C).cuda()
    out = torch.zeros(dm.dmet_emb_eri_bytes(desc, 0) // 8, dtype=torch.float64, device="cuda")
    plan = dm.dmet_emb_plan(desc, stream=torch.cuda.current_stream().cuda_stream)
    try:
        dm.dmet_emb_wait_limit(plan, 2_000_000, test_withhold_loads=True)
        dm.dmet_emb_eri(plan, [Ld], [[Cd]], [[out]])
        st, _ = dm.dmet_emb_status(plan, 0)
        assert st == B.DMET_ERR_TIMEOUT
        msg = dm.dmet_emb_last_error()
        assert "expired" in msg
        # the expired waits are the loaded-stage wait (4) and the accumulator-ready wait (8)
        flags = int(msg.split("flags 0x")[1].split(":")[0], 16)
        assert flags & 4 and flags & 8 and not flags & 32
        # reported once, then the plan runs normally with the default limit
        dm.dmet_emb_wait_limit(plan, 0)
        dm.dmet_emb_eri(plan, [Ld], [[Cd]], [[out]])
        st, _ = dm.dmet_emb_status(plan, 0)
        assert st == B.DMET_OK
    finally:
        dm.dmet_emb_destroy(plan)
    ref = oracle.pack_s8(oracle.embedded_eri(L, C, spec.mesh).real)
    assert rel_fro(out.cpu().numpy(), ref) < 1e-6
