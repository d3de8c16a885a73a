"""The pair schedule of the resident-block Jacobi kernel (ttm_jres.cuh), emulated on the host:
with blocks of B = 8 columns, a round-robin tournament over the blocks (block rounds), the
pairs inside each block at the first block round of a sweep (B - 1 inner rounds of B/2 + B/2
pairs) and the B^2 cross pairs at every block round (column i of the first block with column
(i + s) mod B of the second), every column pair is visited exactly once per sweep and no column
appears twice in an inner round (the rounds' pairs are disjoint), for ragged n and for plan
upper bounds above the realised n. The index arithmetic mirrors the kernel's (jr_pair, the
block columns, the skip of columns beyond n and of the padded block)."""

from collections import Counter

import pytest

B = 8


def rr_pair(k, r, i):
    if i == 0:
        return k - 1, r
    return (r + i) % (k - 1), (r - i + k - 1) % (k - 1)


def sweep_pairs(n, n_ub):
    nb_ub = (n_ub + B - 1) // B
    nbp_ub = nb_ub + (nb_ub & 1)
    nb = (n + B - 1) // B
    nbp = nb + (nb & 1)
    seen = Counter()
    for r in range(nbp_ub - 1):
        for i in range(nbp_ub // 2):
            if i >= nbp // 2 or r >= nbp - 1:
                continue
            P, Q = rr_pair(nbp, r, i)
            col = [(P * B + c if P < nb and P * B + c < n else -1) for c in range(B)] + \
                  [(Q * B + c if Q < nb and Q * B + c < n else -1) for c in range(B)]
            rounds = []
            if r == 0:
                for s in range(B - 1):
                    rnd = []
                    for w in range(B):
                        h = 0 if w < B // 2 else B
                        p, q = rr_pair(B, s, w % (B // 2))
                        rnd.append((p + h, q + h))
                    rounds.append(rnd)
            for s in range(B):
                rounds.append([(w, B + (w + s) % B) for w in range(B)])
            for rnd in rounds:
                local = [c for pq in rnd for c in pq]
                assert len(set(local)) == len(local)          # disjoint pairs in an inner round
                for p, q in rnd:
                    if col[p] >= 0 and col[q] >= 0:
                        seen[frozenset((col[p], col[q]))] += 1
    return seen


@pytest.mark.parametrize("n", list(range(1, 41)) + [63, 64, 65, 127, 128, 129, 255, 257, 512, 1000, 1024])
def test_every_pair_once_per_sweep(n):
    for n_ub in (n, n + 13):
        seen = sweep_pairs(n, n_ub)
        assert len(seen) == n * (n - 1) // 2
        assert all(v == 1 for v in seen.values())
