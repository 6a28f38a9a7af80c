"""Values the paper prints, checked against the oracle's data layout."""
import os

import numpy as np

from oracle.fem import Tables, energy_mass, jacobians
from oracle.mesh import Mesh
from paper_2112_07075_b300 import inputs

HERE = os.path.dirname(__file__)


def _read(name):
    out = {}
    for line in open(os.path.join(HERE, "golden", name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = int(v)
    return out


def test_table1_storage_example():
    g = _read("table1_storage.txt")
    d, p, ne = g["dim"], g["order"], g["elements"]
    n = round(ne ** (1.0 / d))
    m = Mesh(inputs.box_vertices(d, n), d, n, p)
    T = Tables(d, p, p)
    detJ = np.linalg.det(jacobians(T, m.gather(m.x0)))
    pa = detJ * T.w[None, :]                        # quadrature data D of B^T D B
    fa = energy_mass(T, detJ)                       # dense element matrices
    assert m.NE == ne
    assert pa.size == g["partial_assembly_values"]
    assert fa.size == g["full_assembly_values"]
