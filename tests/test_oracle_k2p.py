"""K2P (Section 5.4) in the oracle, on CPU: pruning the next iteration's
k-CNA lists with the previous iteration's pruning reused keeps exactly the
lists of plain pruning (the C oracle) with fewer occlusion checks; a wrong
premise (previous lists that were not the pruning of the previous
candidates) changes the result, so the equality is not vacuous."""
import numpy as np
import pytest

import oracle
import synthetic


def _iteration_inputs(n=500, K=16, R=16, L=32, alpha=66.0):
    D, _, _ = synthetic.workload(1, n=n, nq=1)
    C1, _ = oracle.knn(D, K)
    off1 = np.arange(n + 1, dtype=np.int64) * K
    N1, deg1 = oracle.prune(D, off1, C1.ravel(), R, alpha)
    uoff, uids = oracle.reverse_union(N1, deg1)
    G, gdeg = oracle.prune(D, uoff, uids, R, alpha)
    G, gdeg, _ = oracle.connect(D, G, gdeg, oracle.medoid(D))
    C2 = oracle.acquire(D, G, gdeg, L)
    return D, C1, N1, C2


@pytest.mark.parametrize("alpha", [66.0, 60.0])
def test_k2p_keeps_the_plain_lists_with_fewer_checks(alpha):
    D, C1, N1, C2 = _iteration_inputs(alpha=alpha)
    n, R, L = D.shape[0], 16, C2.shape[1]
    nbr, deg, reused, plain = oracle.prune_k2p(D, C1, N1, C2, R, alpha)
    ref, rdeg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * L, C2.ravel(), R, alpha)
    assert (deg == rdeg).all() and (nbr == ref).all()
    assert reused < plain and reused <= 0.9 * plain, (reused, plain)


def test_k2p_premise_matters():
    D, C1, N1, C2 = _iteration_inputs()
    n, R, L = D.shape[0], 16, C2.shape[1]
    ref, rdeg = oracle.prune(D, np.arange(n + 1, dtype=np.int64) * L, C2.ravel(), R, 66.0)
    # claim every previous candidate was kept: pairs that did occlude are skipped
    nbr, deg, _, _ = oracle.prune_k2p(D, C1, C1, C2, R, 66.0)
    assert (deg != rdeg).any() or (nbr != ref).any()
