"""The seeded input recipes both paths read (no GPU): the indentation state
(bottom clamped, spherical-cap u_z on the top face, one-signed eta noise in
the admissible simplex of Sec. 2.3), the parity-test states, the batch
sizes and the direction vectors. The cap is checked against its closed form:
with R = (a^2 + d^2) / (2 d) the prescribed u_z is -d at the centre and 0 on
the rim r = a."""
import numpy as np
import pytest

from paper_2011_08802_gb300 import inputs


def _grid(mesh):
    X, Y, Z = mesh.node_grid()
    flat = lambda a: a.reshape(-1)  # node order i + (nx+1)(j + (ny+1)k), z-major arrays
    return flat(X), flat(Y), flat(Z)


@pytest.mark.parametrize("n, step", [(8, 1), (12, 5), (16, 10)])
def test_indentation_state(n, step):
    st = inputs.config_indentation(n, seed=5, step=step)
    m = st.mesh
    x, y, z = _grid(m)
    eta = st.U[3:9]
    assert eta.min() >= 0.0 and eta.max() < 1e-3                 # one-signed noise
    assert (1.0 - eta.sum(axis=0)).min() > 0.99                    # eta_0 >= 0: inside the simplex
    np.testing.assert_array_equal(st.Un[3:9], eta)                 # eta_n = eta
    assert not st.Un[0:3].any()
    mask = st.mask.astype(bool)
    assert not mask[3:9].any()                                     # order parameters are never prescribed
    bottom = np.isclose(z, 0.0)
    assert mask[0:3, bottom].all() and not mask[0:2, ~bottom].any()
    # the cap: u_z prescribed on top nodes with r <= a = 0.3 L, nowhere else above the bottom
    top = np.isclose(z, m.Lz)
    r = np.hypot(x - m.Lx / 2, y - m.Ly / 2)
    a = 0.3 * m.Lx
    cap = top & (r <= a + 1e-12 * m.Lx)
    np.testing.assert_array_equal(mask[2] & ~bottom, cap)
    d = 0.02 * m.Lz * step / 10
    R = (a * a + d * d) / (2 * d)
    np.testing.assert_allclose(st.U[2, cap], -(d - (R - np.sqrt(R * R - r[cap] ** 2))), rtol=0, atol=1e-14)
    centre = cap & (r < 1e-12)
    if centre.any():
        assert st.U[2, centre] == pytest.approx(-d, abs=1e-15)
    assert np.abs(st.U[2, cap]).max() <= d + 1e-15
    assert not st.U[0:2].any() and not st.U[2, ~cap].any()


def test_cap_vanishes_on_its_rim():
    mesh = inputs.Mesh(10, 10, 4, 20.0, 20.0, 8.0)
    a, d = 6.0, 0.5
    idx, uz = inputs.cap_displacement(mesh, d, a)
    x, y, _ = _grid(mesh)
    r = np.hypot(x[idx] - 10.0, y[idx] - 10.0)
    rim = np.isclose(r, a)
    assert rim.any()
    np.testing.assert_allclose(uz[rim], 0.0, atol=1e-13)
    assert uz.min() == pytest.approx(-d)


def test_indentation_state_is_seeded():
    s1 = inputs.config_indentation(8, seed=5, step=1)
    s2 = inputs.config_indentation(8, seed=5, step=1)
    s3 = inputs.config_indentation(8, seed=6, step=1)
    np.testing.assert_array_equal(s1.U, s2.U)
    assert not np.array_equal(s1.U[3:9], s3.U[3:9])


@pytest.mark.parametrize("top", [True, False])
def test_random_state(top):
    st = inputs.config_random(7, 5, 3, seed=31, eta_lo=-0.04, eta_hi=0.32, Lx=14.0, Ly=10.0, Lz=6.0, top=top)
    m = st.mesh
    x, y, z = _grid(m)
    eta = st.U[3:9]
    assert eta.min() == pytest.approx(-0.04) and eta.max() == pytest.approx(0.32)
    # u = (z / Lz) g: zero on the bottom; the largest nodal difference quotient is max_grad
    assert not st.U[0:3, np.isclose(z, 0.0)].any()
    u = st.U[0:3].reshape(3, m.nz + 1, m.ny + 1, m.nx + 1)
    hx, hy, hz = m.h
    gmax = max(np.abs(np.diff(u, axis=ax)).max() / h for ax, h in ((3, hx), (2, hy), (1, hz)))
    assert gmax == pytest.approx(0.04, rel=1e-12)
    mask = st.mask.astype(bool)
    assert mask[0:3, np.isclose(z, 0.0)].all()
    assert mask[0:3, np.isclose(z, m.Lz)].all() == top
    assert not mask[3:9].any()


def test_smooth_state_lies_in_the_simplex():
    st = inputs.config_smooth(8, seed=1)
    eta = st.U[3:9]
    assert eta.min() > 0.0 and (1.0 - eta.sum(axis=0)).min() > 0.0


def test_batch_sizes():
    ns, depths = inputs.batch_sizes(64, seed=4)
    assert len(ns) == len(depths) == 64
    assert min(ns) >= 8 and max(ns) <= 24 and len(set(ns)) > 8
    assert min(depths) >= 0.005 and max(depths) <= 0.03
    assert (ns, depths) == inputs.batch_sizes(64, seed=4)


def test_direction_vectors_vanish_on_dirichlet_dofs():
    st = inputs.config_indentation(8, seed=5, step=3)
    v = inputs.direction_vectors(st, 16, seed=3)
    assert v.shape == (16,) + st.U.shape
    assert not v[:, st.mask.astype(bool)].any()
    assert np.abs(v[:, ~st.mask.astype(bool)]).min() > 0.0
