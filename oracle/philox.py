"""Philox4x64-10 counter-based generator, written from its published definition.

Test infrastructure only (see ``oracle/__init__.py``).

Definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 3): a 256-bit counter (c0, c1, c2, c3) of 64-bit words
and a 128-bit key (k0, k1) go through 10 rounds.  One round multiplies c0 and
c2 by two fixed 64-bit constants, keeps both 128-bit products as (hi, lo) and
outputs (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); between rounds the key is
bumped by two Weyl constants (the golden ratio and sqrt(3)-1 in 64-bit fixed
point).  The paper itself does not fix a generator; the noise draws of the
method (Eqs. 1-2, the Monte-Carlo unravelling of the depolarizing channels) are
keyed by this counter so that every implementation reproduces them draw for
draw.
"""

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

TAG_NOISE = 0      # Pauli occurrence and type at one noise site
TAG_MEASURE = 1    # uniform for one ancilla measurement
TAG_READOUT = 3    # uniform for one final data-qubit Z measurement
TAG_TWIRL = 4      # occurrence of one twirled coherent term (site field: factor << 24 | site)


def philox4x64_10(counter, key):
    """Return the four 64-bit output words for ``counter`` (4 ints) and ``key`` (2 ints)."""
    c0, c1, c2, c3 = (int(x) & MASK64 for x in counter)
    k0, k1 = (int(x) & MASK64 for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform53(word):
    """Map a 64-bit word to [0, 1) with 53 bits: (word >> 11) * 2^-53 (exact in FP64)."""
    return (int(word) >> 11) * (1.0 / 9007199254740992.0)


def draw(seed, traj, rnd, step, site, tag):
    """Counter layout: (trajectory index, round, (step << 32) | physical site, stream tag); key (seed, 0)."""
    ctr = (traj, rnd, ((step & 0xFFFFFFFF) << 32) | (site & 0xFFFFFFFF), tag)
    return philox4x64_10(ctr, (seed, 0))
