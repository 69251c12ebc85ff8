"""Linear stability of the rest state on uniform rectangular cells, built from
the oracle's equilibrium (Eq. 19) and the BGK update (Eq. 11) on a doubly
periodic lattice: modes independent of j are never amplified, while on cells
of aspect ratio 2 or more the D2Q21 equilibrium amplifies j-dependent modes
(its populations go negative when g^22 << 1).  D2Q9 is neutral throughout.
This is why symmetric grids are kept exactly independent of j."""
import numpy as np
import pytest

import clbm_inputs as I
from oracle import oracle as O


def _radius(Q, aspect, tau, kys, nk=12):
    n1 = 8
    g = O.Grid(Q, n1, 4, O.PLANAR, edges=I.uniform_edges(n1), step2=float(aspect))
    gi = g.node_geometry(3, 1)["ginv"]
    c, w, _, _, T0 = O.lattice(Q)
    c = c.astype(float)
    h = 1e-6
    zero = np.zeros(2)
    # derivative of f^eq at rest (rho = 1, U = Ut = 0) w.r.t. rho and U (Ut = U)
    d_rho = np.array([(g.feq(a, 1 + h, zero, zero, gi) - g.feq(a, 1 - h, zero, zero, gi)) / (2 * h)
                      for a in range(Q)])
    d_u = np.zeros((Q, 2))
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        d_u[:, k] = [(g.feq(a, 1.0, e, e, gi) - g.feq(a, 1.0, -e, -e, gi)) / (2 * h) for a in range(Q)]
    # perturbation dN -> moments (J = 1): drho = sum dN, dU = sum c dN
    E = np.outer(d_rho, np.ones(Q)) + d_u @ c.T
    best = 0.0
    for kx in np.linspace(0, np.pi, nk):
        for ky in kys:
            D = np.diag(np.exp(-1j * (c[:, 0] * kx + c[:, 1] * ky)))
            A = ((1 - 1 / tau) * np.eye(Q) + E / tau) @ D
            best = max(best, np.abs(np.linalg.eigvals(A)).max())
    return best


@pytest.mark.parametrize("Q", [9, 21])
@pytest.mark.parametrize("aspect", [1.0, 2.0, 4.0])
def test_j_independent_modes_are_never_amplified(Q, aspect):
    for tau in (1.0, 0.6):
        assert _radius(Q, aspect, tau, kys=[0.0]) <= 1 + 1e-9


@pytest.mark.parametrize("aspect", [1.0, 4.0])
def test_d2q9_is_neutral_for_all_modes(aspect):
    assert _radius(9, aspect, 0.8, kys=np.linspace(0, np.pi, 12)) <= 1 + 1e-9


def test_d2q21_amplifies_j_dependent_modes_on_anisotropic_cells():
    kys = np.linspace(0, np.pi, 12)
    assert _radius(21, 1.0, 1.0, kys) <= 1 + 1e-9
    r2 = _radius(21, 2.0, 1.0, kys)
    r4 = _radius(21, 4.0, 1.0, kys)
    assert r2 > 1.05 and r4 > r2
    assert _radius(21, 2.0, 0.6, kys) > r2  # stronger at smaller tau
