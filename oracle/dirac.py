"""Oracle: explicit Dirac matrices and traces with contracted Lorentz indices.

TEST INFRASTRUCTURE ONLY (see the package header).

Conventions of Sec. II: metric g = diag(1, -1, -1, -1) and
gamma^mu gamma^nu + gamma^nu gamma^mu = 2 g^{mu nu}.  The Dirac
representation is used; the on-shell electron momentum is P = (1, 0, 0, 0)
(units m = 1), so Pslash = gamma^0 and P^2 = m^2 = 1.

A trace is given as a list of elements, each either a numeric 4x4 matrix or
('g', label); every label occurs exactly twice and the pair is summed over
with the metric, i.e. gamma^nu ... gamma_nu.  The sum is carried out by
explicit summation over the index values, left to right, keeping one 4x4
matrix per assignment of the currently open indices.

Pinned by textbook identities in the tests (Tr 1 = 4, gamma^nu gamma_nu = 4,
gamma^nu a b c gamma_nu = -2 c b a, trace of four gammas).
"""
import numpy as np

_I2 = np.eye(2)
_Z2 = np.zeros((2, 2))
_SX = np.array([[0, 1], [1, 0]], complex)
_SY = np.array([[0, -1j], [1j, 0]])
_SZ = np.array([[1, 0], [0, -1]], complex)
GAMMA = [np.block([[_I2, _Z2], [_Z2, -_I2]]).astype(complex)] + \
        [np.block([[_Z2, s], [-s, _Z2]]) for s in (_SX, _SY, _SZ)]
METRIC = np.array([1.0, -1.0, -1.0, -1.0])
ONE = np.eye(4, dtype=complex)
PSLASH = GAMMA[0].copy()
GAMMA_UP = np.stack(GAMMA)                                  # gamma^nu
GAMMA_DN = np.stack([METRIC[n] * GAMMA[n] for n in range(4)])  # gamma_nu


def trace(elements):
    """Trace of a product with contracted labels (explicit index sums)."""
    open_labels = []
    state = ONE.copy()                 # shape (4,)*len(open_labels) + (4, 4)
    for el in elements:
        if isinstance(el, tuple) and el[0] == 'g':
            lab = el[1]
            if lab in open_labels:
                ax = open_labels.index(lab)
                st = np.moveaxis(state, ax, 0)          # (4, ..., 4, 4)
                acc = st[0] @ GAMMA_UP[0]
                for nu in range(1, 4):
                    acc = acc + st[nu] @ GAMMA_UP[nu]
                state = acc
                open_labels.pop(ax)
            else:
                state = np.stack([state @ GAMMA_DN[nu] for nu in range(4)], axis=-3)
                open_labels.append(lab)
        else:
            state = state @ el
    assert not open_labels, "unpaired label"
    return np.trace(state)
