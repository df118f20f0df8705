"""Which transformed pairs Algorithm 1 needs, and which of them real-space-real inputs make redundant.

Algorithm 1 (section 2.1) loops over every aux momentum and, inside, over every
momentum-conserving pair; in the q = k2 - k1 labelling the pairs of q are (k1, k1 + q)
for every k1 (momentum conservation of Eq. "density fitting").

With real B and real orbitals (section 2.1: bottom-up local orbitals are real), two
identities hold: Hermiticity L^{k2,k1}_{P,nu mu} = conj(L^{k1,k2}_{P,mu nu}) and time
reversal L^{-k1,-k2} = conj(L^{k1,k2}), C^{-k} = conj(C^k). Their composition maps the pair
(k1, k1+q) to (-k1-q, -k1), which has the same q and contributes the transpose of the
first pair's transformed block. So per q only one k1 of each orbit {k1, -k1-q} is needed
(the fixed points k1 = -k1-q count half), and L^q = s (Z + Z^T) with Z the sum over those
representatives. The factor of -q is the complex conjugate of the factor of q, so only
q <= -q is contracted, with weight 2 (weight 1 when q = -q).
"""
import numpy as np

from .mesh import k_add, k_neg


def schedule(mesh, real):
    nk = int(np.prod(mesh))
    k2_of = np.array([[k_add(k1, q, mesh) for k1 in range(nk)] for q in range(nk)], dtype=np.int32)
    neg = np.array([k_neg(k, mesh) for k in range(nk)], dtype=np.int32)
    q_weight = np.ones(nk, dtype=np.int32)
    n_rep = np.zeros(nk, dtype=np.int32)
    rep_k1 = np.zeros((nk, nk), dtype=np.int32)
    rep_half = np.zeros((nk, nk), dtype=np.int32)
    for q in range(nk):
        if real:
            q_weight[q] = 1 if q == neg[q] else (2 if q < neg[q] else 0)
            reps = []
            for k1 in range(nk):
                partner = k_neg(k_add(k1, q, mesh), mesh)
                if k1 <= partner:
                    reps.append((k1, int(k1 == partner)))
        else:
            reps = [(k1, 0) for k1 in range(nk)]
        n_rep[q] = len(reps)
        for r, (k1, h) in enumerate(reps):
            rep_k1[q, r] = k1
            rep_half[q, r] = h
    return {"k2_of": k2_of, "neg": neg, "q_weight": q_weight, "n_rep": n_rep, "rep_k1": rep_k1,
            "rep_half": rep_half}
