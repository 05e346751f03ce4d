"""D3Q19 velocity set, weights and opposite directions (oracle copy).

The paper only fixes D3Q19 with 19 PDFs per node, one resting and 18 moving,
so 18 neighbour accesses are indirect (Sect. 2 and Sect. 4, "Loop Balance").
The ordering below is the convention this project uses throughout:
direction 0 rests, 1..6 are the axis directions (+x, -x, +y, -y, +z, -z),
7..18 the face diagonals in opposite pairs; the opposite of 2k-1 is 2k.
Weights are the standard D3Q19 ones (1/3, 1/18, 1/36), c_s^2 = 1/3.
"""
import numpy as np

C = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0],
    [0, 1, 0], [0, -1, 0],
    [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0],
    [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1],
    [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1],
    [0, 1, -1], [0, -1, 1],
], dtype=np.int64)

Q = 19


def _opposites():
    inv = np.zeros(Q, dtype=np.int64)
    for i in range(Q):
        for k in range(Q):
            if np.all(C[k] == -C[i]):
                inv[i] = k
    return inv


INV = _opposites()


def _weights():
    w = np.zeros(Q)
    for i in range(Q):
        n2 = int((C[i] ** 2).sum())
        w[i] = {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[n2]
    return w


W = _weights()
