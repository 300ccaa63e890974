"""Ties built on purpose for the decision-margin tests (shared by the
oracle and GPU tests): one atom inside the root cube [0, 2]^3, and the
isovalue c set to that cube's own lower bound L or to the field at a
lattice vertex, so that the margin of that decision is zero."""
import numpy as np

import oracle

ONE_ATOM = (np.array([[0.3, 0.2, 0.1]]), np.array([1.5]))


def tie_on_bound():
    """c equal to the lower bound L of the root cube [0, 2]^3 (one atom
    inside it: the tensor does not depend on c)."""
    xyz, r = ONE_ATOM
    A, cnt = oracle.cube_tensor(xyz, r, 0.5, 1.0, np.zeros(3), 2.0)
    assert cnt == 1
    return float(oracle.bounds(A)[0])


def tie_on_vertex():
    """c equal to the field at the lattice vertex (1, 1, 1)."""
    xyz, r = ONE_ATOM
    return float(oracle.field(xyz, r, 0.5, 1.0, np.array([[1.0, 1.0, 1.0]]))[0])
