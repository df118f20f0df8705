"""k-mesh index arithmetic on a Gamma-centred mesh (section 2.2: Gamma-centred meshes).

A k-point n = (n1, n2, n3), 0 <= n_d < N_d, has the C-order index
(n1*N2 + n2)*N3 + n3. Sums and negations of k-points are taken modulo the mesh,
i.e. modulo reciprocal lattice vectors (the n*b of Eq. "density fitting").
"""


def k_triplet(k, mesh):
    n1, n2, n3 = mesh
    return (k // (n2 * n3), (k // n3) % n2, k % n3)


def k_index(t, mesh):
    n1, n2, n3 = mesh
    return ((t[0] % n1) * n2 + (t[1] % n2)) * n3 + (t[2] % n3)


def k_add(k1, k2, mesh):
    a, b = k_triplet(k1, mesh), k_triplet(k2, mesh)
    return k_index((a[0] + b[0], a[1] + b[1], a[2] + b[2]), mesh)


def k_neg(k, mesh):
    a = k_triplet(k, mesh)
    return k_index((-a[0], -a[1], -a[2]), mesh)
