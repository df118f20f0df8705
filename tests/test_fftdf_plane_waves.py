"""The library's FFTDF plane-wave tables (dmet_fftdf_plane_waves, host-only, Appendix B) against the
oracle's Coulomb kernel, and the opposite-plane-wave map against vector arithmetic. No GPU needed."""
import numpy as np
import pytest

import oracle.fftdf as of
from oracle.mesh import k_neg, k_triplet
import paper_1909_08596_gb300 as dm
from paper_1909_08596_gb300 import binding as B

LAT = ((2.0, 0.0, 0.0), (0.3, 2.2, 0.0), (0.1, 0.2, 2.5))
CASES = [((1, 1, 1), (4, 4, 4)), ((2, 1, 1), (4, 4, 4)), ((3, 1, 1), (3, 5, 3)), ((3, 3, 1), (3, 3, 5)),
         ((2, 2, 1), (3, 4, 3)), ((4, 3, 2), (5, 2, 3))]


@pytest.mark.parametrize("mesh,grid", CASES)
def test_plane_wave_tables_match_oracle(mesh, grid):
    nk = int(np.prod(mesh))
    b = 2.0 * np.pi * np.linalg.inv(np.asarray(LAT)).T
    for q in range(nk):
        m, v, opp = dm.dmet_fftdf_plane_waves(mesh, q, grid, LAT)
        want = of.coulomb_kernel(q, mesh, LAT, grid).ravel()
        np.testing.assert_allclose(v, want, rtol=1e-14, atol=0)
        # m_d = j_d mod g_d
        j = np.stack(np.meshgrid(*[np.arange(g) for g in grid], indexing="ij"), -1).reshape(-1, 3)
        assert np.array_equal(np.mod(m, grid), j)
        # opposite: -(q + G) = (-q) + G' up to a supercell reciprocal vector on Nyquist axes, and a permutation
        assert sorted(opp.tolist()) == list(range(int(np.prod(grid))))
        mq, _, _ = dm.dmet_fftdf_plane_waves(mesh, k_neg(q, mesh), grid, LAT)
        t = np.asarray(k_triplet(q, mesh)) / np.asarray(mesh)
        tn = np.asarray(k_triplet(k_neg(q, mesh), mesh)) / np.asarray(mesh)
        s = (m + t) * np.asarray(mesh)                 # supercell frequencies of q + G
        sp = (mq[opp] + tn) * np.asarray(mesh)         # those of the opposite plane waves
        big = np.asarray(mesh) * np.asarray(grid)
        assert np.all(np.mod(np.round(s + sp), big) == 0)
        odd = big % 2 == 1
        assert np.all(np.round(s + sp)[:, odd] == 0)


def test_plane_wave_tables_reject_bad_arguments():
    for args in (((0, 1, 1), 0, (4, 4, 4), LAT), ((2, 1, 1), 2, (4, 4, 4), LAT),
                 ((2, 1, 1), 0, (4, 0, 4), LAT), ((2, 1, 1), 0, (4, 4, 4), ((1, 0, 0), (2, 0, 0), (0, 0, 1)))):
        with pytest.raises(B.DmetError) as e:
            dm.dmet_fftdf_plane_waves(*args)
        assert e.value.status == B.DMET_ERR_INVALID_ARG
