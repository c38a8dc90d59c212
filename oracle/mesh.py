"""Structured macro mesh, macro-element lattice and trace numbering (oracle).

Test infrastructure only. The conventions below are the library's published
data layout (the C header states the same rules); they are restated here from
that description, not shared as code.

Macro mesh (Sec. 5.1 for d = 2: N = 2 n^2 macro-triangles). The unit square is
cut into n x n squares; square (i, j) = [x_i, x_{i+1}] x [y_j, y_{j+1}] with
x_i = i / n is split by its "/" diagonal into
  t = 0 (lower-right): v0 = (x_{i+1}, y_j), v1 = (x_{i+1}, y_{j+1}), v2 = (x_i, y_j)
  t = 1 (upper-left) : v0 = (x_i, y_{j+1}), v1 = (x_i, y_j),         v2 = (x_{i+1}, y_{j+1})
Element id e = 2 (j n + i) + t. Vertices are counter-clockwise, v0 is the
right-angle vertex, local edge k is opposite v_k and runs from v_{k+1} to
v_{k+2} (indices mod 3).

Macro-element lattice (Sec. 3.2): the reference triangle (0,0),(1,0),(0,1) is
mapped affinely by x = v0 + xi (v1 - v0) + eta (v2 - v0). With P = m p, the
C0 P_p nodes are (a/P, b/P), a + b <= P, numbered b-major, a fastest:
  node(a, b) = b (P + 1) - b (b - 1) / 2 + a.
Sub-triangles (m^2, uniform subdivision), in units of 1/m:
  upright  (si, sj), si + sj <= m - 1: A = (si, sj),       B = (si+1, sj),   C = (si, sj+1)
  inverted (si, sj), si + sj <= m - 2: A = (si+1, sj+1),   B = (si, sj+1),   C = (si+1, sj)
enumerated upright first (sj outer, si inner), then inverted (sj outer, si
inner).

Skeleton and trace numbering (Sec. 2.2, 3.2): global vertex (i, j) has id
j (n + 1) + i; every edge is oriented from its lower to its higher vertex id
(+x, +y or +diagonal). Interior edges are the trace unknowns (all-Dirichlet
boundary):
  diagonal   D(i, j), 0 <= i, j < n       : j n + i
  horizontal H(i, j), y = y_j, 1 <= j < n  : n^2 + (j - 1) n + i
  vertical   V(i, j), x = x_i, 1 <= i < n  : n^2 + n (n - 1) + j (n - 1) + (i - 1)
Each edge carries P + 1 trace dofs (C0 P_p on its m sub-edges) at equispaced
points along its orientation; global dof = edge * (P + 1) + s.
Boundary (Dirichlet) edges: bottom H(i, 0) -> i, top H(i, n) -> n + i,
left V(0, j) -> 2 n + j, right V(n, j) -> 3 n + j.
Element edges: t = 0: (D(i,j), flip), (H(i,j), same), (V(i+1,j), same);
               t = 1: (D(i,j), same), (H(i,j+1), flip), (V(i,j), flip).
"""
import numpy as np


class StructuredMesh:
    def __init__(self, n, m, p):
        if n < 1 or m < 1 or p < 1:
            raise ValueError("n, m, p must be >= 1")
        self.n, self.m, self.p = n, m, p
        self.P = m * p
        self.N = 2 * n * n
        self.Q = (self.P + 1) * (self.P + 2) // 2
        self.P1 = self.P + 1
        self.n_t = 3 * self.P1
        self.n_int_edges = n * n + 2 * n * (n - 1)
        self.n_bnd_edges = 4 * n
        self.N_tr = self.n_int_edges * self.P1

    # ---------------------------------------------------------------- geometry
    def vertices(self, e):
        n = self.n
        sq, t = divmod(e, 2)
        j, i = divmod(sq, n)
        x0, x1 = i / n, (i + 1) / n
        y0, y1 = j / n, (j + 1) / n
        if t == 0:
            v = [(x1, y0), (x1, y1), (x0, y0)]
        else:
            v = [(x0, y1), (x0, y0), (x1, y1)]
        return np.array(v, dtype=np.float64)

    # ----------------------------------------------------------------- lattice
    def node(self, a, b):
        P = self.P
        return b * (P + 1) - b * (b - 1) // 2 + a

    def lattice_ref(self):
        """Reference coordinates (xi, eta) of the Q lattice nodes, in node order."""
        P = self.P
        pts = np.empty((self.Q, 2))
        for b in range(P + 1):
            for a in range(P + 1 - b):
                pts[self.node(a, b)] = (a / P, b / P)
        return pts

    def sub_triangles(self):
        """List of (A, B, C) vertex triples in units of 1/m, in the published order."""
        m = self.m
        out = []
        for sj in range(m):
            for si in range(m - sj):
                out.append(((si, sj), (si + 1, sj), (si, sj + 1)))
        for sj in range(m - 1):
            for si in range(m - 1 - sj):
                out.append(((si + 1, sj + 1), (si, sj + 1), (si + 1, sj)))
        return out

    def sub_nodes(self, tri):
        """Lattice node indices of the P_p Lagrange nodes of one sub-triangle.

        Returns (alphas, nodes): alphas[k] = (alpha_A, alpha_B, alpha_C) with sum p,
        nodes[k] = lattice index of the point (alpha_A A + alpha_B B + alpha_C C) / p.
        """
        p = self.p
        (Aa, Ab), (Ba, Bb), (Ca, Cb) = tri
        alphas, nodes = [], []
        for aC in range(p + 1):
            for aB in range(p + 1 - aC):
                aA = p - aB - aC
                la = aA * Aa + aB * Ba + aC * Ca       # in units of 1/(m p)
                lb = aA * Ab + aB * Bb + aC * Cb
                alphas.append((aA, aB, aC))
                nodes.append(self.node(la, lb))
        return alphas, nodes

    # ---------------------------------------------------------------- skeleton
    def diag_edge(self, i, j):
        return j * self.n + i

    def horiz_edge(self, i, j):
        n = self.n
        if j == 0:
            return ("bnd", i)
        if j == n:
            return ("bnd", n + i)
        return ("int", n * n + (j - 1) * n + i)

    def vert_edge(self, i, j):
        n = self.n
        if i == 0:
            return ("bnd", 2 * n + j)
        if i == n:
            return ("bnd", 3 * n + j)
        return ("int", n * n + n * (n - 1) + j * (n - 1) + (i - 1))

    def element_edges(self, e):
        """[(kind, index, flip)] for local edges 0, 1, 2 of element e."""
        n = self.n
        sq, t = divmod(e, 2)
        j, i = divmod(sq, n)
        d = ("int", self.diag_edge(i, j))
        if t == 0:
            return [d + (1,), self.horiz_edge(i, j) + (0,), self.vert_edge(i + 1, j) + (0,)]
        return [d + (0,), self.horiz_edge(i, j + 1) + (1,), self.vert_edge(i, j) + (1,)]

    def boundary_edge_endpoints(self, b):
        """Endpoints (start, end) of Dirichlet edge b, in its global orientation."""
        n = self.n
        side, k = divmod(b, n)
        h = 1.0 / n
        if side == 0:
            return np.array([k * h, 0.0]), np.array([(k + 1) * h, 0.0])
        if side == 1:
            return np.array([k * h, 1.0]), np.array([(k + 1) * h, 1.0])
        if side == 2:
            return np.array([0.0, k * h]), np.array([0.0, (k + 1) * h])
        return np.array([1.0, k * h]), np.array([1.0, (k + 1) * h])

    def element_dof_map(self, e):
        """For each of the n_t element-local trace dofs: (kind, global index).

        kind 'int' -> index into the unknown trace vector; 'bnd' -> index into
        the Dirichlet trace array [n_bnd_edges * (P + 1)].
        """
        P1, P = self.P1, self.P
        out = []
        for (kind, idx, flip) in self.element_edges(e):
            for s_loc in range(P1):
                s = P - s_loc if flip else s_loc
                out.append((kind, idx * P1 + s))
        return out
