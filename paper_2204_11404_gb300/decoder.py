"""Host-side decoder: detection events, minimum-weight perfect matching, logical readout.

Sec. III.B: detection events are the XOR of the syndromes of adjacent rounds;
the error positions are estimated by minimum-weight perfect matching; the
logical value after correction decides failure.  The paper does not give the
graph or weights, so this module uses the plain reading.
- The space-time graph has one node per (event layer, Z-stabilizer).
- Unit-weight space edges join stabilizers that share a data qubit (one X error
  before both of their gates on it).
- Unit-weight diagonal edges join the later-gated stabilizer in one layer with
  the earlier-gated one in the next layer (one X error between their two gates
  on that qubit: the later gate sees it this round, the earlier one next round).
- Unit-weight time edges join the same stabilizer in consecutive layers (one
  measurement error).
- A data qubit in only one Z-stabilizer is an edge to the boundary.
- The last layer of events compares the last measured syndrome with the
  Z-stabilizer parities of the final data readout.

Only Z-stabilizers are decoded, because the experiment measures logical Z.
Logical Z is Z on the first data row (surface code) or on the whole line
(repetition code, Fig. 2).  A correction chain flips the logical when it
crosses that support an odd number of times.

Edge weights are 1 by default.  Log-likelihood weights w = log((1 - p) / p) can be
set from edge probabilities, for instance those estimated from the detection events
themselves (estimate_edge_probabilities: the two-point correlation of independent
mechanisms, Spitz et al., Adv. Quantum Technol. 1, 1800012 (2018)); shortest paths are
then found by Dijkstra instead of breadth-first search.

The matching is exact (dynamic programming over subsets of defects) up to
MAX_EXACT defects.  Beyond that it falls back to greedy pairing of the closest
defects, and the count of such trajectories is reported.
"""
import heapq
from collections import deque
from functools import lru_cache

import numpy as np

MAX_EXACT = 16


def _stabilizers(d):
    """Z-stabilizers in serial order (same rule as the library's program builder): list of
    (support sorted, {data qubit: gate slot}) with slots clockwise from the top-right corner."""
    zs = []
    for r in range(-1, d):
        for c in range(-1, d):
            if (r + c) % 2:
                continue
            corners = [(r, c + 1), (r + 1, c + 1), (r + 1, c), (r, c)]   # TR, BR, BL, TL
            cells = [(a, b) for (a, b) in corners if 0 <= a < d and 0 <= b < d]
            if len(cells) == 4 or (len(cells) == 2 and (c == -1 or c == d - 1) and not (r == -1 or r == d - 1)):
                slots = {a * d + b: i for i, (a, b) in enumerate(corners) if 0 <= a < d and 0 <= b < d}
                zs.append(((c, -r), sorted(slots), slots))
    zs.sort(key=lambda t: t[0])
    return [(sup, slots) for _, sup, slots in zs]


def _repetition_stabilizers(d):
    """Z_k Z_{k+1} in line order, gate order q_{k+1} then q_k (as the library builds them)."""
    return [([k, k + 1], {k + 1: 0, k: 1}) for k in range(d - 1)]


class Decoder:
    def __init__(self, d, code="surface"):
        self.d, self.code = d, code
        st = _repetition_stabilizers(d) if code == "repetition" else _stabilizers(d)
        self.zs = [sup for sup, _ in st]
        self.slots = [sl for _, sl in st]
        self.nz = len(self.zs)
        # X-stabilizers come first in the syndrome rows (the repetition code has none)
        self.nx = 0 if code == "repetition" else self.nz
        nd = d if code == "repetition" else d * d
        owners = [[] for _ in range(nd)]
        for k, sup in enumerate(self.zs):
            for q in sup:
                owners[q].append(k)
        self.owners = owners
        self.row = set(range(d))               # logical Z support
        self.fallbacks = 0
        self._graphs = {}
        self._edges = {}
        self._w = {}

    def edges(self, layers):
        """Edges of the space-time graph of `layers` event layers: list of (u, v, parity, kind), node
        (e, k) = e * nz + k, boundary node layers * nz, kind "space", "diag", "boundary" or "time"."""
        if layers in self._edges:
            return self._edges[layers]
        nz, B = self.nz, layers * self.nz
        out = []
        for q, ks in enumerate(self.owners):
            par = 1 if q in self.row else 0
            for e in range(layers):
                if len(ks) == 2:
                    out.append((e * nz + ks[0], e * nz + ks[1], par, "space"))
                    if e + 1 < layers:
                        early, late = sorted(ks, key=lambda k: self.slots[k][q])
                        out.append((e * nz + late, (e + 1) * nz + early, par, "diag"))
                elif len(ks) == 1:
                    out.append((e * nz + ks[0], B, par, "boundary"))
        for e in range(layers - 1):
            for k in range(nz):
                out.append((e * nz + k, (e + 1) * nz + k, 0, "time"))
        self._edges[layers] = out
        return out

    def _graph(self, layers):
        """Adjacency of the space-time graph: node -> [(node, parity, edge index)]."""
        if layers in self._graphs:
            return self._graphs[layers]
        B = layers * self.nz
        adj = [[] for _ in range(B + 1)]
        for i, (u, v, par, _) in enumerate(self.edges(layers)):
            adj[u].append((v, par, i))
            adj[v].append((u, par, i))
        self._graphs[layers] = (adj, B)
        return adj, B

    def set_edge_probabilities(self, layers, p):
        """Log-likelihood weights log((1 - p_e) / p_e) for the edges of `layers` layers (in the order
        of edges(layers)); p is clipped to [1e-12, 0.5 - 1e-12]."""
        p = np.clip(np.asarray(p, dtype=np.float64), 1e-12, 0.5 - 1e-12)
        if p.shape != (len(self.edges(layers)),):
            raise ValueError("one probability per edge")
        self._w[layers] = np.log((1.0 - p) / p)

    def clear_weights(self):
        self._w.clear()

    def event_matrix(self, syndromes, data_bits):
        """0/1 detection events [n][layers * nz] of n trajectories with the same number of rounds."""
        layers = len(syndromes[0])
        X = np.zeros((len(syndromes), layers * self.nz), dtype=np.uint8)
        for t, (s, b) in enumerate(zip(syndromes, data_bits)):
            for e, k in self.detection_events(s, b):
                X[t, e * self.nz + k] = 1
        return X

    def estimate_edge_probabilities(self, events):
        """Edge probabilities from detection events [n][layers * nz], each edge an independent
        mechanism that flips its two nodes.  A node pair (i, j) is flipped together with probability
        p = 1/2 - sqrt(1/4 - (<x_i x_j> - <x_i><x_j>) / (1 - 2<x_i> - 2<x_j> + 4<x_i x_j>)).  A node's
        boundary edges take what its one-point rate leaves: 1 - 2<x_i> = prod over the node's edges
        of (1 - 2 p_e).  Parallel edges share their pair's probability equally."""
        X = np.asarray(events, dtype=np.float64)
        layers = X.shape[1] // self.nz
        E = self.edges(layers)
        m = X.mean(axis=0)
        groups = {}
        for i, (u, v, _, kind) in enumerate(E):
            groups.setdefault((min(u, v), max(u, v)) if kind != "boundary" else (u, -1), []).append(i)
        p = np.zeros(len(E))
        rest = np.ones(X.shape[1])   # product of (1 - 2 p_e) over each node's non-boundary edges
        for (u, v), idx in groups.items():
            if v < 0:
                continue
            xij = float(np.mean(X[:, u] * X[:, v]))
            den = 1.0 - 2.0 * m[u] - 2.0 * m[v] + 4.0 * xij
            q = 0.0
            if den > 0:
                q = 0.5 - np.sqrt(max(0.0, 0.25 - (xij - m[u] * m[v]) / den))
            q = min(max(q, 0.0), 0.5 - 1e-12)
            each = 0.5 * (1.0 - (1.0 - 2.0 * q) ** (1.0 / len(idx)))
            p[idx] = each
            rest[u] *= 1.0 - 2.0 * q
            rest[v] *= 1.0 - 2.0 * q
        for (u, _), idx in groups.items():
            if _ >= 0:
                continue
            ratio = (1.0 - 2.0 * m[u]) / rest[u] if rest[u] > 0 else 1.0
            qb = min(max(0.5 * (1.0 - ratio), 0.0), 0.5 - 1e-12)
            p[idx] = 0.5 * (1.0 - (1.0 - 2.0 * qb) ** (1.0 / len(idx)))
        return p

    def _bfs(self, adj, B, src):
        n = len(adj)
        dist = [-1] * n
        par = [0] * n
        dist[src] = 0
        dq = deque([src])
        while dq:
            u = dq.popleft()
            if u == B and src != B:
                continue                       # a chain ends at the boundary
            for v, pq, _ in adj[u]:
                if dist[v] < 0:
                    dist[v] = dist[u] + 1
                    par[v] = par[u] ^ pq
                    dq.append(v)
        return dist, par

    def _dijkstra(self, adj, B, src, w):
        n = len(adj)
        dist = [float("inf")] * n
        par = [0] * n
        dist[src] = 0.0
        heap = [(0.0, src)]
        while heap:
            du, u = heapq.heappop(heap)
            if du > dist[u] or (u == B and src != B):
                continue                       # stale entry, or a chain that ends at the boundary
            for v, pq, ei in adj[u]:
                nd = du + float(w[ei])
                if nd < dist[v]:
                    dist[v] = nd
                    par[v] = par[u] ^ pq
                    heapq.heappush(heap, (nd, v))
        return dist, par

    def detection_events(self, syndromes, data_bits):
        """syndromes [R+1][d^2-1] (row 0 = init), data_bits [d^2] -> list of (round, z index)."""
        s = np.asarray(syndromes, dtype=np.uint8)[:, self.nx:]     # rows 0 (init) .. R
        final = np.array([np.bitwise_xor.reduce(np.asarray(data_bits, dtype=np.uint8)[sup]) for sup in self.zs],
                         dtype=np.uint8)
        full = np.vstack([s, final[None, :]])
        ev = full[1:] ^ full[:-1]
        return [(int(r), int(k)) for r, k in zip(*np.nonzero(ev))]

    def _match(self, defects, layers):
        n = len(defects)
        if n == 0:
            return 0
        adj, B = self._graph(layers)
        weights = self._w.get(layers)
        nodes = [e * self.nz + k for e, k in defects]
        w = np.zeros((n, n), dtype=np.float64)
        p = np.zeros((n, n), dtype=np.uint8)
        wb = np.zeros(n, dtype=np.float64)
        pb = np.zeros(n, dtype=np.uint8)
        for i, u in enumerate(nodes):
            dist, par = self._bfs(adj, B, u) if weights is None else self._dijkstra(adj, B, u, weights)
            for j, v in enumerate(nodes):
                w[i, j], p[i, j] = dist[v], par[v]
            wb[i], pb[i] = dist[B], par[B]
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
            out = (c + float(wb[i]), q ^ int(pb[i]))
            m = rest
            while m:
                j = (m & -m).bit_length() - 1
                m &= m - 1
                c2, q2 = best(rest & ~(1 << j))
                cand = (c2 + float(w[i, j]), q2 ^ int(p[i, j]))
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

    def correction_parity(self, defects, layers):
        """Parity of the matched correction across the logical Z support, for defects (layer, k)."""
        return self._match(list(defects), layers)

    def logical_failure(self, syndromes, data_bits, raw_logical):
        """1 if the decoded logical Z differs from the prepared |0_L> (Sec. III.B)."""
        layers = len(syndromes)                # event layers: rounds 1..R and the final readout
        return int(raw_logical) ^ self._match(self.detection_events(syndromes, data_bits), layers)

    def logical_error_rate(self, syndromes, data_bits, raw_logical):
        f = [self.logical_failure(s, b, l) for s, b, l in zip(syndromes, data_bits, raw_logical)]
        return float(np.mean(f)) if f else 0.0


def count_failures(dec, syndromes, data_bits, raw_logical):
    """(failures with unit weights, failures with log-likelihood weights) over n trajectories of the
    same rounds.  The weights come from edge probabilities estimated on these trajectories' own
    detection events; the decoder's weights are left as they were."""
    layers = len(syndromes[0])
    saved = dec._w.pop(layers, None)
    unit = sum(dec.logical_failure(s, b, l) for s, b, l in zip(syndromes, data_bits, raw_logical))
    dec.set_edge_probabilities(layers, dec.estimate_edge_probabilities(dec.event_matrix(syndromes, data_bits)))
    weighted = sum(dec.logical_failure(s, b, l) for s, b, l in zip(syndromes, data_bits, raw_logical))
    dec._w.pop(layers, None)
    if saved is not None:
        dec._w[layers] = saved
    return int(unit), int(weighted)
