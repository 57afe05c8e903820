"""CHP stabilizer-tableau simulator (Aaronson & Gottesman, Phys. Rev. A 70, 052328 (2004)).

Test infrastructure only (see ``oracle/__init__.py``).  Pins the state-vector
oracle on Pauli-only noise: with every coherent term off, the circuit of
Sec. III.A is Clifford, so each measurement is either deterministic or a fair
coin, and with the same uniforms (outcome 1 iff u < 1/2 for a coin) the two
simulators must agree bit for bit.

Clifford forms used (each equal to the named matrix up to a global phase,
checked in the tests): Rz(pi/2) ~ S, Rx(pi/2) ~ H S H, Rx^dagger(pi/2) ~ H S^3 H,
Rzx(pi/2) with Z on a and X on b ~ H_b CNOT_ab S_b CNOT_ab H_b.
"""
import numpy as np

from . import gates as G


class Tableau:
    def __init__(self, n):
        self.n = n
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros(2 * n + 1, dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1          # destabilizers X_i
            self.z[n + i, i] = 1      # stabilizers Z_i

    # gates (applied to all 2n rows; the scratch row is excluded)
    def h(self, a):
        x, z = self.x[:-1], self.z[:-1]
        self.r[:-1] ^= x[:, a] & z[:, a]
        x[:, a], z[:, a] = z[:, a].copy(), x[:, a].copy()

    def s(self, a):
        x, z = self.x[:-1], self.z[:-1]
        self.r[:-1] ^= x[:, a] & z[:, a]
        z[:, a] ^= x[:, a]

    def cnot(self, a, b):
        x, z = self.x[:-1], self.z[:-1]
        self.r[:-1] ^= x[:, a] & z[:, b] & (x[:, b] ^ z[:, a] ^ 1)
        x[:, b] ^= x[:, a]
        z[:, a] ^= z[:, b]

    def pauli(self, a, code):
        x, z = self.x[:-1], self.z[:-1]
        if code == 1:
            self.r[:-1] ^= z[:, a]
        elif code == 3:
            self.r[:-1] ^= x[:, a]
        elif code == 2:
            self.r[:-1] ^= x[:, a] ^ z[:, a]

    @staticmethod
    def _g(x1, z1, x2, z2):
        x1, z1, x2, z2 = (v.astype(np.int64) for v in (x1, z1, x2, z2))
        return np.where((x1 == 1) & (z1 == 1), z2 - x2,
                        np.where((x1 == 1) & (z1 == 0), z2 * (2 * x2 - 1),
                                 np.where((x1 == 0) & (z1 == 1), x2 * (1 - 2 * z2), 0)))

    def _rowsum(self, h, i):
        tot = 2 * int(self.r[h]) + 2 * int(self.r[i]) + int(self._g(self.x[i], self.z[i], self.x[h], self.z[h]).sum())
        self.r[h] = 0 if tot % 4 == 0 else 1
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def measure(self, a, u, forced=-1):
        """Z measurement of qubit a.  Returns (outcome, P(1)) with P(1) in {0, 1/2, 1}."""
        n = self.n
        ps = [p for p in range(n, 2 * n) if self.x[p, a]]
        if ps:
            p = ps[0]
            for i in range(2 * n):
                if i != p and self.x[i, a]:
                    self._rowsum(i, p)
            self.x[p - n], self.z[p - n], self.r[p - n] = self.x[p].copy(), self.z[p].copy(), self.r[p]
            self.x[p] = 0
            self.z[p] = 0
            self.z[p, a] = 1
            out = forced if forced >= 0 else (1 if u < 0.5 else 0)
            self.r[p] = out
            return out, 0.5
        sc = 2 * n
        self.x[sc] = 0
        self.z[sc] = 0
        self.r[sc] = 0
        for i in range(n):
            if self.x[i, a]:
                self._rowsum(sc, i + n)
        out = int(self.r[sc])
        if forced >= 0 and forced != out:
            raise RuntimeError("forced outcome has zero probability")
        return out, float(out)


def _close_up_to_phase(a, b):
    k = np.argmax(np.abs(b))
    if abs(b.flat[k]) < 1e-12:
        return False
    ph = a.flat[k] / b.flat[k]
    return abs(abs(ph) - 1) < 1e-12 and np.allclose(a, ph * b, atol=1e-12)


def apply_op(tab, op):
    """Apply one op of circuit.Trajectory to the tableau (Clifford ops only)."""
    kind = op[0]
    if kind == "U1":
        q, m = op[1], op[2]
        for code in (1, 2, 3):
            if _close_up_to_phase(m, G.PAULI[code]):
                tab.pauli(q, code)
                return
        if _close_up_to_phase(m, G.H):
            tab.h(q)
        elif _close_up_to_phase(m, G.RZ90):
            tab.s(q)
        elif _close_up_to_phase(m, G.RX90):
            tab.h(q); tab.s(q); tab.h(q)
        elif _close_up_to_phase(m, G.RX90DG):
            tab.h(q); tab.s(q); tab.s(q); tab.s(q); tab.h(q)
        else:
            raise ValueError("non-Clifford one-qubit op")
    elif kind == "U2":
        a, b, m = op[1], op[2], op[3]
        for ca in range(4):                  # a product of Paulis (twirled two-qubit terms)
            for cb in range(4):
                if (ca or cb) and _close_up_to_phase(m, np.kron(G.PAULI[ca], G.PAULI[cb])):
                    if ca:
                        tab.pauli(a, ca)
                    if cb:
                        tab.pauli(b, cb)
                    return
        if _close_up_to_phase(m, G.CNOT):
            tab.cnot(a, b)
        elif _close_up_to_phase(m, G.RZX90):
            tab.h(b); tab.cnot(a, b); tab.s(b); tab.cnot(a, b); tab.h(b)
        else:
            raise ValueError("non-Clifford two-qubit op")
    else:
        raise ValueError("measurements are handled by run_ops")


def run_ops(tab, ops):
    outs, p1s = [], []
    for op in ops:
        if op[0] == "M":
            q, u, forced, reset = op[1], op[2], op[3], op[4]
            o, p = tab.measure(q, u, forced)
            if reset and o:
                tab.pauli(q, 1)
            outs.append(o)
            p1s.append(p)
        else:
            apply_op(tab, op)
    return outs, p1s
