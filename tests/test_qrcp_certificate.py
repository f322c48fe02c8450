"""The multi-pivot certificate of the single-precision sketch QRCP, checked on
the CPU in FP64: taking up to four pivots per grid barrier never changes the
greedy pivot order of Alg. 1.

The device kernel splits the n columns into G contiguous slabs.  At each
barrier every slab publishes its best column and a bound (its second-best
trailing norm); after the winner's reflector, a candidate (a slab's best
above every bound) whose updated trailing norm is strictly above every bound
is the next greedy pivot, because trailing norms only shrink under the
reflectors; the test repeats with each new reflector, up to four pivots.  This
test replays that rule with numpy Householder reflectors and compares the
pivots with the oracle's partial QRCP (exact recomputed norms, one pivot at a
time), and checks that the rule does save barriers.
"""
import numpy as np
import pytest

import oracle


def _house(x):
    alpha = x[0]
    nx = np.linalg.norm(x)
    beta = -nx if alpha >= 0 else nx
    v = x / (alpha - beta)
    v[0] = 1.0
    return v, (beta - alpha) / beta


def _certified_qrcp(B, k, G, maxp):
    """Pivots and barrier count of the slab certificate (maxp pivots per barrier)."""
    s, n = B.shape
    W = B.copy()
    sel = np.zeros(n, dtype=bool)
    edges = [(n * b) // G for b in range(G + 1)]
    piv, j, barriers = [], 0, 0
    while j < k:
        nrm = np.sum(W[j:, :] ** 2, axis=0)
        nrm[sel] = -1.0
        best, bidx, second = [], [], []
        for b in range(G):
            seg = nrm[edges[b]:edges[b + 1]]
            order = np.argsort(-seg, kind="stable")  # ties: lowest index first
            best.append(seg[order[0]])
            bidx.append(edges[b] + order[0])
            second.append(seg[order[1]] if len(order) > 1 else -1.0)
        bound = max(second)
        top = max(range(G), key=lambda b: (best[b], -bidx[b]))
        taken = [bidx[top]]
        cands = [bidx[b] for b in range(G) if best[b] > bound and b != top]
        barriers += 1
        while True:
            c = taken[-1]
            p = j + len(taken) - 1
            v, tau = _house(W[p:, c].copy())
            W[p:, :] -= tau * np.outer(v, v @ W[p:, :])
            if len(taken) == maxp or j + len(taken) >= k or not cands:
                break
            q = j + len(taken)
            nn = {c2: float(np.sum(W[q:, c2] ** 2)) for c2 in cands}
            c2 = max(cands, key=lambda x: (nn[x], -x))
            if not (nn[c2] > bound and nn[c2] > 0.0):
                break
            taken.append(c2)
            cands.remove(c2)
        for c in taken:
            sel[c] = True
        piv += taken
        j += len(taken)
    return piv[:k], barriers


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_certificate_keeps_the_greedy_order(seed):
    rng = np.random.default_rng(seed)
    s, n, k, G = 30, 400, 25, 16
    # column norms spread over two decades, as in a sketch of a decaying spectrum
    B = rng.standard_normal((s, n)) * np.exp(rng.uniform(-2.3, 0.0, n))[None, :]
    perm, _, _ = oracle.qrcp(B, k)
    greedy = list(perm[:k])
    one, bars1 = _certified_qrcp(B, k, G, 1)
    two, bars2 = _certified_qrcp(B, k, G, 2)
    four, bars4 = _certified_qrcp(B, k, G, 4)
    assert one == greedy and bars1 == k
    assert two == greedy and four == greedy
    assert bars4 < bars2 < bars1
