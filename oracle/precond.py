"""Face-block preconditioner of the condensed trace system (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Not in the paper, which left-preconditions GMRES with D^-1 (Sec. 6.1), D_f
the trace-trace face block of the unreduced system. This preconditioner takes
the exact diagonal face blocks of the condensed operator itself: with S the
matrix of Eq. (global_problem) and I_f the trace dofs of interior face f,
S_ff = S[I_f, I_f], and GMRES runs on P S x = P g with P = blockdiag(S_ff)^-1.
Written out from that definition: the blocks are read out of the assembled S
and inverted (or solved with) densely. The transposed operator S^T of the
adjoint has the face blocks S_ff^T.
"""
import numpy as np


def face_blocks(S, eoff):
    """S_ff for every face f, whose dofs are eoff[f] .. eoff[f + 1] - 1."""
    return [np.array(S[eoff[f]:eoff[f + 1], eoff[f]:eoff[f + 1]]) for f in range(len(eoff) - 1)]


def face_block_inverse(S, eoff):
    """blockdiag(S_ff)^-1 as a dense matrix of the shape of S."""
    P = np.zeros_like(S)
    for f, B in enumerate(face_blocks(S, eoff)):
        sl = slice(eoff[f], eoff[f + 1])
        P[sl, sl] = np.linalg.inv(B)
    return P


def apply_face_blocks(S, eoff, y):
    """z with z[I_f] = S_ff^-1 y[I_f] on every face (dense solves)."""
    z = np.empty_like(y)
    for f, B in enumerate(face_blocks(S, eoff)):
        sl = slice(eoff[f], eoff[f + 1])
        z[sl] = np.linalg.solve(B, y[sl])
    return z
