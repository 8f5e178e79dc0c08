"""CPU oracle of the Newton-step solve of the finite-strain multivariant
phase-field model (plain NumPy/SciPy, float64).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import anything from this
package. It shares no code with the CUDA path and never imports it; the two
meet only in the seeded input generators of
``paper_2011_08802_gb300.inputs``, which hold no part of the method.

Modules:
* ``jet``: exact second-order forward-mode differentiation on batches;
* ``qp``: local energy density of Sec. 2 / Eq. PenPot at a quadrature point;
* ``fe``: Q1-hexahedron discretisation, residual, tangent, JVP, direct solve.
"""
