"""Code geometry: data qubits, stabilizers, two-qubit gate order (rotated surface code; the
one-dimensional repetition code of Fig. 2 as a second workload).

Test infrastructure only (see ``oracle/__init__.py``).

* Data qubits (Sec. II.A, Fig. 1a caption, Table I): a d x d grid numbered
  row-major, paper index 1..d^2; here 0-based, data id j = paper index - 1.
* Stabilizers (Table I): plaquettes whose top-left corner sits at (r, c),
  r, c in {-1..d-1}, cover the grid cells (r..r+1, c..c+1).  A plaquette is
  X-type when r + c is odd.  Full (weight-4) plaquettes are all kept; weight-2
  ones are kept on the top/bottom edge for X-type and on the left/right edge
  for Z-type; corner (weight-1) plaquettes are dropped.  Table I lists the
  X-stabilizers by plaquette row (top to bottom, then left to right) and the
  Z-stabilizers by plaquette column (left to right, then bottom to top); that
  listing order is also the serial (delayed) measurement order used here
  (X part of a round, then Z part; Sec. II.B, Fig. 3).
* Two-qubit gate order (Sec. II.A): X-type stabilizers go clockwise from the
  bottom-right corner (BR, BL, TL, TR), Z-type clockwise from the top-right
  corner (TR, BR, BL, TL); a missing corner is a "wait" slot.
* Logical Z: Z on the first data row.  Sec. III.B prints Z1 Z7 Z13 Z19 Z25,
  which anticommutes with X1X2 of Table I, so the printed operator is read as
  a typo for a row of Z operators (any row is equivalent modulo Z-stabilizers).
"""


def data_id(d, r, c):
    return r * d + c


def _plaquettes(d):
    out = []
    for r in range(-1, d):
        for c in range(-1, d):
            cells = [(r, c), (r, c + 1), (r + 1, c), (r + 1, c + 1)]
            inside = [(a, b) for (a, b) in cells if 0 <= a < d and 0 <= b < d]
            kind = "X" if (r + c) % 2 else "Z"
            if len(inside) == 4:
                out.append((kind, r, c))
            elif len(inside) == 2:
                horizontal_edge = r == -1 or r == d - 1
                vertical_edge = c == -1 or c == d - 1
                if kind == "X" and horizontal_edge and not vertical_edge:
                    out.append((kind, r, c))
                if kind == "Z" and vertical_edge and not horizontal_edge:
                    out.append((kind, r, c))
    return out


def _corner(d, r, c):
    if 0 <= r < d and 0 <= c < d:
        return data_id(d, r, c)
    return None


def stabilizers(d):
    """Serial-order list of dicts: kind ('X'/'Z'), slots (4 data ids or None, in gate order),
    support (sorted data ids), and weight.  X-stabilizers first, in Table I order, then Z."""
    xs, zs = [], []
    for kind, r, c in _plaquettes(d):
        tl, tr = _corner(d, r, c), _corner(d, r, c + 1)
        bl, br = _corner(d, r + 1, c), _corner(d, r + 1, c + 1)
        if kind == "X":
            slots = [br, bl, tl, tr]
            xs.append(((r, c), slots))
        else:
            slots = [tr, br, bl, tl]
            zs.append(((c, -r), slots))
    xs.sort(key=lambda t: t[0])
    zs.sort(key=lambda t: t[0])
    out = []
    for kind, lst in (("X", xs), ("Z", zs)):
        for _, slots in lst:
            support = sorted(q for q in slots if q is not None)
            out.append({"kind": kind, "slots": slots, "support": support, "weight": len(support)})
    return out


def logical_z_support(d, code="surface"):
    """Surface code: the first data row.  Repetition code: all d data qubits (Z on every qubit of
    the line, equal to Z on one qubit times stabilizers for odd d)."""
    if code == "repetition":
        return list(range(d))
    return [data_id(d, 0, c) for c in range(d)]


def repetition_stabilizers(d):
    """One-dimensional bit-flip repetition code (Sec. II.B, Fig. 2): d data qubits on a line,
    stabilizers Z_k Z_{k+1}, k = 0..d-2, all Z-type.  Gate order q_{k+1} then q_k, so that
    measuring k = 0, 1, ... one at a time keeps every qubit's gates in time order (qubit k+1 meets
    stabilizer k at the first gate step and stabilizer k+1 at the second): the time-shifted
    circuit of Fig. 2(b).  Slots 3 and 4 of the Z part are waits."""
    return [{"kind": "Z", "slots": [k + 1, k, None, None], "support": [k, k + 1], "weight": 2}
            for k in range(d - 1)]


def code_stabilizers(d, code="surface"):
    if code == "surface":
        return stabilizers(d)
    if code == "repetition":
        return repetition_stabilizers(d)
    raise ValueError("code must be 'surface' or 'repetition'")


def n_data(d, code="surface"):
    return d if code == "repetition" else d * d


def n_stabilizers(d):
    return d * d - 1
