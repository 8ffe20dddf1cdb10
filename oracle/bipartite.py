"""Agent-location (JUNE-style) contact structure for the oracle (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``.

GradABM-JUNE (Sec. 6) represents contacts as a heterogeneous graph of agents and
locations.  Two agents interact through every location they share, so the model
on the agent-location graph is the one-hop model of Sec. 3.1 on the agent graph
with pair weights W_ij = sum_l w_il w_jl (i != j): the force of infection
lambda_i = R S_i (1/Dbar) sum_l w_il sum_{j at l, j != i} w_jl x_j is Eq. 3 with
those weights, and Dbar is W's mean weighted degree.  ``expand`` writes W out
(the plain definition), so the oracle's one-hop forward and adjoint apply as they
stand.  Only small populations can be expanded: W has a clique per location.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Expanded:
    n: int
    rowptr: np.ndarray   # uint64 [n+1], row i lists the agents j it meets
    col: np.ndarray      # uint32 [nnz]
    w: np.ndarray        # float32 [nnz]  W_ij, rounded once from FP64
    age: np.ndarray
    w64: np.ndarray      # float64 [nnz]  W_ij before rounding

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def incidence(bip) -> sp.csr_matrix:
    """The n x n_loc incidence matrix B with B[i, l] = w_il (FP64)."""
    rowptr = np.asarray(bip.rowptr, np.int64)
    return sp.csr_matrix((np.asarray(bip.w, np.float64), np.asarray(bip.loc, np.int64), rowptr),
                         shape=(bip.n, bip.n_loc))


def expand(bip) -> Expanded:
    """W = B B^T without its diagonal: W_ij = sum over shared locations of w_il w_jl."""
    B = incidence(bip)
    W = (B @ B.T).tocsr()
    W.setdiag(0.0)
    W.eliminate_zeros()
    W.sort_indices()
    return Expanded(n=bip.n, rowptr=W.indptr.astype(np.uint64), col=W.indices.astype(np.uint32),
                    w=W.data.astype(np.float32), age=np.asarray(bip.age, np.uint8), w64=W.data.copy())


def mean_weighted_degree(bip) -> float:
    """Dbar of W from the incidence alone: (1/n) sum_l [(sum_i w_il)^2 - sum_i w_il^2]."""
    B = incidence(bip)
    col_sum = np.asarray(B.sum(axis=0)).ravel()
    col_sq = np.asarray(B.multiply(B).sum(axis=0)).ravel()
    return float((col_sum ** 2 - col_sq).sum() / bip.n)
