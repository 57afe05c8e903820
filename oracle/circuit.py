"""One Monte-Carlo trajectory of the noisy syndrome-extraction experiment, as an op list.

Test infrastructure only (see ``oracle/__init__.py``).

Protocol (Sec. III.B): data start in |0>; one noise-free round whose
measurements are forced to the zero syndrome projects onto the code state;
then ``rounds`` noisy rounds; then every data qubit is measured in Z, in index
order.  Each round is an X part (steps 1-6) then a Z part (steps 7-11), which
gives the 11 steps per cycle of Sec. III.D.

Gate sets (Sec. III.A):
* "cnot": X-stabilizer = H(anc), CNOT(anc -> data) x4, H(anc); Z-stabilizer =
  CNOT(data -> anc) x4.  Steps 6 and 11 are idle for data qubits.
* "cr": H before -> Rx^dagger(pi/2), H after -> Rx(pi/2), CNOT -> Rzx(pi/2)
  with Z on the control side; data get Rx(pi/2)^{nX(q)} at step 6 and
  Rz(pi/2)^{nZ(q)} at step 11, nX/nZ = number of X/Z stabilizers holding q.
  With Rzx, a weight-2 stabilizer's raw ancilla bit is the inverted parity, so
  its syndrome bit is raw XOR 1 (weight 4: raw).

Noise at each step (Eqs. 1-2), per qubit in its active window (data: all
steps; X ancilla: steps 1-6; Z ancilla: steps 7-11): a qubit pair in a
two-qubit gate gets the two-qubit depolarizing channel with p2 (one of the 15
non-identity pairs, uniformly: Eq. 2 read with its weights normalised), a
qubit in a one-qubit gate gets Eq. 1 with p1, an idle ("wait") qubit gets
Eq. 1 with p_idle.  Coherent terms (Sec. III.A): after every Rx/Rx^dagger an
extra R_X(theta_rx), after every Rz an extra R_Z(theta_rz), after every Rzx an
extra exp(-i theta_rzx Z(x)X / 2), after every two-qubit gate exp(-i phi_zz
Z(x)Z); not on waits.  Per round, before step 1, R_Z(round_rz) then
R_X(round_rx) on every data qubit.  Order on a qubit within a step: gate,
coherent terms, Pauli.

Layouts (Sec. II.B): "reduced" has d^2 data qubits plus one ancilla (bit d^2)
reused by every stabilizer, run one stabilizer circuit at a time in the
serial order; every data qubit keeps its own step clock so its idle noise and
corrections are applied in its own time order.  "unreduced" keeps all d^2-1
ancillas (bits d^2 + k) and runs the circuit step by step.  Both consume the
same random draws: noise sites are keyed by (round, step, physical qubit) with
ancilla k numbered d^2 + k, a two-qubit gate's site is its data qubit.

Twirled variant (twirl = 1; Sec. III.A: a coherent term whose coherence is
destroyed, e.g. by twirling, acts as a stochastic Pauli error): every
coherent term R_A(theta) is replaced by the Pauli A with probability
sin^2(theta/2), and the crosstalk exp(-i phi Z(x)Z) by Z(x)Z with probability
sin^2(phi).  Each such term is a draw of its own (tag 4, site field
factor << 24 | site, factor = index of the term on that site in that step:
0..3 the one-qubit terms after Rx/Rz factors, 4 the Rzx term, 5 the ZZ term,
6 / 7 the round-start R_Z / R_X).

Over-rotation sign (Sec. III.A gives exp(-i c sqrt(p) A) for every rotation gate): by default
the extra rotation has the same sign after every gate, Rx^dagger included.  With
overrot_follows = 1 (a flagged variant) the extra rotation after Rx^dagger(pi/2), the only
negative-angle rotation gate of the schedule (X-ancilla preparation at step 1), is R_X(-theta_rx):
the magnitude of every gate's angle grows.

Draws (Philox4x64-10, counter (trajectory, round, step<<32 | site, tag)):
occurrence iff (w0 >> 11) 2^-53 < p; Eq. 1 Pauli index = ((w1 >> 32) * 3 >> 32)
-> X, Y, Z; Eq. 2 pair index k = ((w1 >> 32) * 15 >> 32) + 1, ancilla Pauli
k >> 2, data Pauli k & 3 (0=I, 1=X, 2=Y, 3=Z).  Measurement uniforms use w0 the
same way (tag 1, step 0, site = physical ancilla; final readout tag 3, round
rounds+1, site = data qubit).
"""
import numpy as np

from . import gates as G
from .lattice import code_stabilizers, logical_z_support, n_data
from .philox import draw, uniform53, TAG_NOISE, TAG_MEASURE, TAG_READOUT, TAG_TWIRL

NOISE_KEYS = ("p1", "p2", "p_idle", "theta_rx", "theta_rz", "theta_rzx", "phi_zz", "round_rz", "round_rx", "twirl",
              "overrot_follows")


def noise_dict(**kw):
    out = {k: 0.0 for k in NOISE_KEYS}
    for k, v in kw.items():
        if k not in out:
            raise KeyError(k)
        out[k] = float(v)
    return out


class Trajectory:
    """Builds the op list of one trajectory and records the sampled Pauli events."""

    def __init__(self, d, rounds, gates, layout, noise, seed, traj, inject=None, code="surface"):
        if gates not in ("cnot", "cr") or layout not in ("reduced", "unreduced"):
            raise ValueError("bad gate set or layout")
        self.d, self.rounds, self.gates, self.layout, self.code = d, rounds, gates, layout, code
        self.noise = noise_dict(**(noise or {}))
        self.seed, self.traj = seed, traj
        self.nd = n_data(d, code)
        self.stabs = code_stabilizers(d, code)
        self.nstab = len(self.stabs)
        self.n = self.nd + (1 if layout == "reduced" else self.nstab)
        self.inject = inject or []        # (round, step, data qubit, 2x2 matrix), applied after that step's ops
        self.ops = []
        self.events = []                  # sampled Paulis: (round, step, site, pauli code)
        self.twirls = []                  # fired twirled terms: (round, step, site, factor)
        self.meas = []                    # measurement records, in op order
        nx = [0] * self.nd
        nz = [0] * self.nd
        for s in self.stabs:
            for q in s["support"]:
                (nx if s["kind"] == "X" else nz)[q] += 1
        self.nx, self.nz = nx, nz

    # ---- op emitters -------------------------------------------------------------------
    def u1(self, q, m):
        self.ops.append(("U1", q, np.asarray(m, dtype=complex)))

    def u2(self, qa, qb, m):
        self.ops.append(("U2", qa, qb, np.asarray(m, dtype=complex)))

    def anc_qubit(self, k):
        return self.nd if self.layout == "reduced" else self.nd + k

    def e1(self, rnd, t, site, q, p):
        if rnd == 0 or p <= 0.0:
            return
        w = draw(self.seed, self.traj, rnd, t, site, TAG_NOISE)
        if uniform53(w[0]) < p:
            code = (((w[1] >> 32) * 3) >> 32) + 1
            self.events.append((rnd, t, site, code))
            self.u1(q, G.PAULI[code])

    def coherent1(self, rnd, t, site, factor, q, pauli, theta):
        """R_P(theta) on q, or (twirled) the Pauli P with probability sin^2(theta/2)."""
        if not theta:
            return
        if not self.noise["twirl"]:
            self.u1(q, G.rot(pauli, theta))
            return
        w = draw(self.seed, self.traj, rnd, t, (factor << 24) | site, TAG_TWIRL)
        if uniform53(w[0]) < np.sin(theta / 2) ** 2:
            self.twirls.append((rnd, t, site, factor))
            self.u1(q, pauli)

    def coherent2(self, rnd, t, site, factor, qa, qb, pauli2, angle, zz):
        """exp(-i angle/2 P) (Rzx term) or exp(-i angle P) (ZZ term, zz=True) on (qa, qb); twirled:
        the Pauli product with probability sin^2(angle/2) / sin^2(angle)."""
        if not angle:
            return
        if not self.noise["twirl"]:
            self.u2(qa, qb, G.zz_crosstalk(angle) if zz else G.rot(pauli2, angle))
            return
        w = draw(self.seed, self.traj, rnd, t, (factor << 24) | site, TAG_TWIRL)
        prob = np.sin(angle) ** 2 if zz else np.sin(angle / 2) ** 2
        if uniform53(w[0]) < prob:
            self.twirls.append((rnd, t, site, factor))
            self.u2(qa, qb, pauli2)

    def e2(self, rnd, t, site, qa, qd, p):
        if rnd == 0 or p <= 0.0:
            return
        w = draw(self.seed, self.traj, rnd, t, site, TAG_NOISE)
        if uniform53(w[0]) < p:
            k = (((w[1] >> 32) * 15) >> 32) + 1
            a, b = k >> 2, k & 3
            self.events.append((rnd, t, site, 4 * a + b))
            if a:
                self.u1(qa, G.PAULI[a])
            if b:
                self.u1(qd, G.PAULI[b])

    # ---- per-step pieces ---------------------------------------------------------------
    def data_step(self, rnd, q, t):
        """Ops on data qubit q at step t when q is not in a two-qubit gate (t = 0: round start)."""
        nz = self.noise
        noisy = rnd > 0
        if t == 0:
            if noisy:
                self.coherent1(rnd, t, q, 6, q, G.PZ, nz["round_rz"])
                self.coherent1(rnd, t, q, 7, q, G.PX, nz["round_rx"])
        elif self.gates == "cr" and t in (6, 11):
            n_fact = self.nx[q] if t == 6 else self.nz[q]
            base = G.RX90 if t == 6 else G.RZ90
            over = nz["theta_rx"] if t == 6 else nz["theta_rz"]
            pauli = G.PX if t == 6 else G.PZ
            for f in range(n_fact):
                self.u1(q, base)
                if noisy:
                    self.coherent1(rnd, t, q, f, q, pauli, over)
            # no correction gate (a code with no stabilizer of that kind on q): the qubit idles
            self.e1(rnd, t, q, q, nz["p1"] if n_fact else nz["p_idle"])
        else:
            self.e1(rnd, t, q, q, nz["p_idle"])
        for (ri, ti, qi, m) in self.inject:
            if ri == rnd and ti == t and qi == q:
                self.u1(q, m)

    def anc_step(self, rnd, k, t, on_data):
        """Ops of stabilizer k's ancilla at step t; on_data(q, t) is called before a gate on q."""
        nz = self.noise
        noisy = rnd > 0
        s = self.stabs[k]
        a = self.anc_qubit(k)
        site_a = self.nd + k
        if s["kind"] == "X":
            if t in (1, 6):
                if self.gates == "cnot":
                    self.u1(a, G.H)
                else:
                    self.u1(a, G.RX90DG if t == 1 else G.RX90)
                    if noisy:
                        # sign-follows variant: the over-rotation of Rx^dagger turns the same way
                        sgn = -1.0 if (t == 1 and nz["overrot_follows"]) else 1.0
                        self.coherent1(rnd, t, site_a, 0, a, G.PX, sgn * nz["theta_rx"])
                self.e1(rnd, t, site_a, a, nz["p1"])
                return
            slot = t - 2
        else:
            if t == 11:
                self.e1(rnd, t, site_a, a, nz["p_idle"])
                return
            slot = t - 7
        q = s["slots"][slot]
        if q is None:
            self.e1(rnd, t, site_a, a, nz["p_idle"])
            return
        on_data(q, t)
        # (first, second) = (control side, target side)
        first, second = (a, q) if s["kind"] == "X" else (q, a)
        if self.gates == "cnot":
            self.u2(first, second, G.CNOT)
        else:
            self.u2(first, second, G.RZX90)
            if noisy:
                self.coherent2(rnd, t, q, 4, first, second, G.ZX, nz["theta_rzx"], zz=False)
        if noisy:
            self.coherent2(rnd, t, q, 5, first, second, G.ZZ, nz["phi_zz"], zz=True)
        self.e2(rnd, t, q, a, q, nz["p2"])

    def measure_anc(self, rnd, k):
        s = self.stabs[k]
        offset = 1 if (self.gates == "cr" and s["weight"] == 2) else 0
        if rnd == 0:
            u, forced = 0.0, offset
        else:
            u, forced = uniform53(draw(self.seed, self.traj, rnd, 0, self.nd + k, TAG_MEASURE)[0]), -1
        self.ops.append(("M", self.anc_qubit(k), u, forced, 1))
        self.meas.append(("anc", rnd, k, offset, u))

    # ---- schedules ---------------------------------------------------------------------
    def part_indices(self, kind):
        return [k for k, s in enumerate(self.stabs) if s["kind"] == kind]

    def round_reduced(self, rnd):
        clock = [-1] * self.nd

        def flush(q, upto):
            for t in range(clock[q] + 1, upto + 1):
                self.data_step(rnd, q, t)
            clock[q] = upto

        def on_data(q, t):
            flush(q, t - 1)
            clock[q] = t

        for kind, steps, last in (("X", range(1, 7), 6), ("Z", range(7, 12), 11)):
            for k in self.part_indices(kind):
                for t in steps:
                    self.anc_step(rnd, k, t, on_data)
                self.measure_anc(rnd, k)
            for q in range(self.nd):
                flush(q, last)

    def round_unreduced(self, rnd):
        for q in range(self.nd):
            self.data_step(rnd, q, 0)
        for kind, steps in (("X", range(1, 7)), ("Z", range(7, 12))):
            ks = self.part_indices(kind)
            for t in steps:
                busy = set()
                for k in ks:
                    self.anc_step(rnd, k, t, lambda q, tt: busy.add(q))
                for q in range(self.nd):
                    if q not in busy:
                        self.data_step(rnd, q, t)
            for k in ks:
                self.measure_anc(rnd, k)

    def build(self):
        for rnd in range(0, self.rounds + 1):
            if self.layout == "reduced":
                self.round_reduced(rnd)
            else:
                self.round_unreduced(rnd)
        r_final = self.rounds + 1
        for j in range(self.nd):
            u = uniform53(draw(self.seed, self.traj, r_final, 0, j, TAG_READOUT)[0])
            self.ops.append(("M", j, u, -1, 0))
            self.meas.append(("data", r_final, j, 0, u))
        return self

    def readout_start(self):
        """Index into self.ops of the first final-readout measurement."""
        for i, op in enumerate(self.ops):
            if op[0] == "M" and op[4] == 0:
                return i
        return len(self.ops)


def logical_parity(d, data_bits, code="surface"):
    return int(np.bitwise_xor.reduce([int(data_bits[q]) for q in logical_z_support(d, code)]))
