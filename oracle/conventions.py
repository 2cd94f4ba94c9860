"""Dirac-matrix conventions of the oracle.

The paper does not fix a gamma basis.  The oracle uses the chiral basis

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = 1, 2, 3 -> mu = 0, 1, 2)
    gamma_4 = [[0, 1], [1, 0]]                     (mu = 3, the time direction)

so that gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1): spins 0, 1
have chirality +1 and spins 2, 3 chirality -1.  This is what makes the
"nbasis = twice the number of basis vectors" of Sec. 5 a chiral split of each
basis vector into its two spin halves.

sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu].
"""
import numpy as np

PAULI = np.array(
    [[[0, 1], [1, 0]],
     [[0, -1j], [1j, 0]],
     [[1, 0], [0, -1]]],
    dtype=np.complex128,
)


def _gammas() -> np.ndarray:
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    for k in range(3):
        g[k, 0:2, 2:4] = -1j * PAULI[k]
        g[k, 2:4, 0:2] = 1j * PAULI[k]
    g[3, 0:2, 2:4] = np.eye(2)
    g[3, 2:4, 0:2] = np.eye(2)
    return g


GAMMA = _gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def sigma_munu(mu: int, nu: int) -> np.ndarray:
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])


# chirality (0 for +, 1 for -) of each of the 12 fine components s*3 + c
FINE_CHIRALITY = np.array([(d // 3) // 2 for d in range(12)])
