"""Counting formulas of Sec. 5.1 (Tables 1-2), dimension-generic (oracle).

Test infrastructure only.
    N     = d! n^d                          macro-elements
    Q_(d) = C(m p + d, d)                   C0 P_p lattice nodes per d-simplex
    D     = A_d n^d + B_d d n^(d-1) (n - 1) interior faces, (A_2, B_2) = (1, 1),
                                           (A_3, B_3) = (6, 2)
Boundary faces of the structured cube: 2 d n^(d-1) (d-1)! (each boundary facet
of the cube is split like the cube faces of the simplicial mesh).
dof^local  = N (d + 1) Q_(d)   ((q, u) per lattice node, Tables 7 and 9 text)
dof^global = faces * Q_(d-1)   (trace on every face; the 3D tables include
                                the boundary faces)
"""
from math import comb, factorial

_AB = {2: (1, 1), 3: (6, 2)}


def n_macro(d, n):
    return factorial(d) * n ** d


def q_nodes(d, m, p):
    return comb(m * p + d, d)


def interior_faces(d, n):
    A, B = _AB[d]
    return A * n ** d + B * d * n ** (d - 1) * (n - 1)


def boundary_faces(d, n):
    return 2 * d * n ** (d - 1) * factorial(d - 1)


def dof_local(d, n, m, p):
    return n_macro(d, n) * (d + 1) * q_nodes(d, m, p)


def dof_global(d, n, m, p, with_boundary=True):
    faces = interior_faces(d, n) + (boundary_faces(d, n) if with_boundary else 0)
    return faces * q_nodes(d - 1, m, p)
