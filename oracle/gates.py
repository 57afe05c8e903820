"""Gate and noise matrices of the simulated circuit (Sec. III.A).

Test infrastructure only (see ``oracle/__init__.py``).

Convention: R_A(theta) = exp(-i theta A / 2) for a Pauli string A (A^2 = I), so
R_A(theta) = cos(theta/2) I - i sin(theta/2) A.  The native gates are
Rx(pi/2) = exp(-i pi X/4), Rx^dagger(pi/2), Rz(pi/2) = exp(-i pi Z/4) and
Rzx(pi/2) = exp(-i pi Z(x)X/4) (cross-resonance; Z on the control side, X on the
target side).  A two-qubit matrix acts on the local index 2*bit(first) + bit(second).
"""
import numpy as np

I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = [I2, PX, PY, PZ]          # index 0=I, 1=X, 2=Y, 3=Z


def rot(A, theta):
    """exp(-i theta A / 2) for a Pauli (string) matrix A."""
    A = np.asarray(A, dtype=complex)
    return np.cos(theta / 2) * np.eye(A.shape[0], dtype=complex) - 1j * np.sin(theta / 2) * A


ZX = np.kron(PZ, PX)              # Z on the first-listed qubit, X on the second
ZZ = np.kron(PZ, PZ)

RX90 = rot(PX, np.pi / 2)
RX90DG = rot(PX, -np.pi / 2)
RZ90 = rot(PZ, np.pi / 2)
RZX90 = rot(ZX, np.pi / 2)
H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)


def zz_crosstalk(phi):
    """Unintended ZZ interaction exp(-i phi Z(x)Z) after a two-qubit gate."""
    return np.diag(np.exp(-1j * phi * np.diag(ZZ).real)).astype(complex)
