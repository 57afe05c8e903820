"""Host-side decoder: detection events, minimum-weight perfect matching, logical readout.

Sec. III.B: detection events are the XOR of the syndromes of adjacent rounds;
the error positions are estimated by minimum-weight perfect matching; the
logical value after correction decides failure.  The paper does not give the
graph or weights, so this module uses the plain reading.
- The space-time graph has one node per (round, Z-stabilizer).
- Unit-weight edges join stabilizers that share a data qubit (one X error), or
  the same stabilizer in consecutive rounds (one measurement error).
- A data qubit in only one Z-stabilizer is an edge to the boundary.
- The last round of events compares the last measured syndrome with the
  Z-stabilizer parities of the final data readout.

Only Z-stabilizers are decoded, because the experiment measures logical Z.
Logical Z is Z on the first data row.  A correction chain flips the logical
when it crosses that row an odd number of times.

The matching is exact (dynamic programming over subsets of defects) up to
MAX_EXACT defects.  Beyond that it falls back to greedy pairing of the closest
defects, and the count of such trajectories is reported.
"""
from collections import deque
from functools import lru_cache

import numpy as np

MAX_EXACT = 16


def _stabilizers(d):
    """Z-stabilizer supports in serial order (same rule as the library's program builder)."""
    zs = []
    for r in range(-1, d):
        for c in range(-1, d):
            cells = [(a, b) for (a, b) in ((r, c), (r, c + 1), (r + 1, c), (r + 1, c + 1)) if 0 <= a < d and 0 <= b < d]
            if (r + c) % 2:
                continue
            if len(cells) == 4 or (len(cells) == 2 and (c == -1 or c == d - 1) and not (r == -1 or r == d - 1)):
                zs.append(((c, -r), sorted(a * d + b for (a, b) in cells)))
    zs.sort(key=lambda t: t[0])
    return [s for _, s in zs]


class Decoder:
    def __init__(self, d):
        self.d = d
        self.zs = _stabilizers(d)
        self.nz = len(self.zs)
        self.nx = self.nz                      # X-stabilizers come first in the syndrome rows
        nd = d * d
        owners = [[] for _ in range(nd)]
        for k, sup in enumerate(self.zs):
            for q in sup:
                owners[q].append(k)
        B = self.nz                            # boundary node
        adj = [[] for _ in range(self.nz + 1)]
        for q, ks in enumerate(owners):
            if len(ks) == 2:
                adj[ks[0]].append((ks[1], q))
                adj[ks[1]].append((ks[0], q))
            elif len(ks) == 1:
                adj[ks[0]].append((B, q))
                adj[B].append((ks[0], q))
        row = set(range(d))                    # logical Z support
        n = self.nz + 1
        self.dist = np.zeros((n, n), dtype=np.int64)
        self.par = np.zeros((n, n), dtype=np.uint8)
        for s in range(n):
            dist = [-1] * n
            par = [0] * n
            dist[s] = 0
            dq = deque([s])
            while dq:
                u = dq.popleft()
                if u == B and s != B:
                    continue                   # paths do not pass through the boundary
                for v, q in adj[u]:
                    if dist[v] < 0:
                        dist[v] = dist[u] + 1
                        par[v] = par[u] ^ (1 if q in row else 0)
                        dq.append(v)
            self.dist[s] = dist
            self.par[s] = par
        self.boundary = B
        self.z_of_data = owners
        self.fallbacks = 0

    def detection_events(self, syndromes, data_bits):
        """syndromes [R+1][d^2-1] (row 0 = init), data_bits [d^2] -> list of (round, z index)."""
        s = np.asarray(syndromes, dtype=np.uint8)[:, self.nx:]
        final = np.array([np.bitwise_xor.reduce(np.asarray(data_bits, dtype=np.uint8)[sup]) for sup in self.zs],
                         dtype=np.uint8)
        full = np.vstack([s, final[None, :]])
        ev = full[1:] ^ full[:-1]
        return [(int(r), int(k)) for r, k in zip(*np.nonzero(ev))]

    def _match(self, defects):
        n = len(defects)
        if n == 0:
            return 0
        B = self.boundary
        w = np.zeros((n, n), dtype=np.int64)
        p = np.zeros((n, n), dtype=np.uint8)
        for i, (ri, ki) in enumerate(defects):
            for j, (rj, kj) in enumerate(defects):
                w[i, j] = self.dist[ki, kj] + abs(ri - rj)
                p[i, j] = self.par[ki, kj]
        wb = np.array([self.dist[k, B] for _, k in defects], dtype=np.int64)
        pb = np.array([self.par[k, B] for _, k in defects], dtype=np.uint8)
        if n > MAX_EXACT:
            self.fallbacks += 1
            return self._greedy(w, p, wb, pb)

        @lru_cache(maxsize=None)
        def best(mask):
            if mask == 0:
                return (0, 0)
            i = (mask & -mask).bit_length() - 1
            rest = mask & ~(1 << i)
            c, q = best(rest)
            out = (c + int(wb[i]), q ^ int(pb[i]))
            m = rest
            while m:
                j = (m & -m).bit_length() - 1
                m &= m - 1
                c2, q2 = best(rest & ~(1 << j))
                cand = (c2 + int(w[i, j]), q2 ^ int(p[i, j]))
                if cand[0] < out[0]:
                    out = cand
            return out

        return best((1 << n) - 1)[1]

    @staticmethod
    def _greedy(w, p, wb, pb):
        n = len(wb)
        left = set(range(n))
        flip = 0
        while left:
            i = min(left)
            left.remove(i)
            j = min(left, key=lambda t: w[i, t], default=None)
            if j is not None and w[i, j] < wb[i] + wb[j]:
                left.remove(j)
                flip ^= int(p[i, j])
            else:
                flip ^= int(pb[i])
        return flip

    def logical_failure(self, syndromes, data_bits, raw_logical):
        """1 if the decoded logical Z differs from the prepared |0_L> (Sec. III.B)."""
        return int(raw_logical) ^ self._match(self.detection_events(syndromes, data_bits))

    def logical_error_rate(self, syndromes, data_bits, raw_logical):
        f = [self.logical_failure(s, b, l) for s, b, l in zip(syndromes, data_bits, raw_logical)]
        return float(np.mean(f)) if f else 0.0
