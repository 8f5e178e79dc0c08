"""Oracle evaluations split over element chunks and run by spawned worker
processes, one per host core (test infrastructure). The oracle's residual
and tangent are sums over elements (Sec. 3.4), so each worker evaluates the
contributions of its chunk and the parent adds them up. Workers are
spawned, never forked, so that none inherits a CUDA context, and run with one
BLAS thread each."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _residual_chunk(args):
    mesh, U, Un, mask, tau, material, elems = args
    from oracle import fe, qp
    from paper_2011_08802_gb300 import inputs
    st = inputs.State(mesh, U, Un, mask, tau, material)
    disc = fe.Discretisation(mesh, elements=elems)
    return fe.residual(disc, st, qp.material_from(material, tau))


def _rows_chunk(args):
    mesh, U, Un, mask, tau, material, x, elems, nodes = args
    from oracle import fe, qp
    from paper_2011_08802_gb300 import inputs
    st = inputs.State(mesh, U, Un, mask, tau, material)
    disc = fe.Discretisation(mesh, elements=elems)
    mat = qp.material_from(material, tau)
    d = fe.qp_derivatives(disc, st, mat, order=2)
    # K x + R of the chunk's elements; Dirichlet rows (identity in K, zero in
    # R) are left at 0 here and added once by the caller
    y = fe.jvp(disc, st, x, d) + fe.residual(disc, st, mat, d)
    y[mask.astype(bool)] = 0.0
    return y[:, nodes]


class OraclePool:
    """A spawned process pool for chunked oracle evaluations:

        with OraclePool() as pool:
            Rs = pool.residuals([state_a, state_b])
    """

    def __init__(self, processes: int | None = None):
        self.processes = processes or len(os.sched_getaffinity(0))
        self.pool = None

    def __enter__(self):
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        os.environ.update({k: "1" for k in _THREAD_VARS})
        try:
            self.pool = mp.get_context("spawn").Pool(self.processes)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()

    def _chunks(self, n_elems: int, parts: int):
        return [c for c in np.array_split(np.arange(n_elems), parts) if c.size]

    def residuals(self, states) -> list[np.ndarray]:
        """The oracle residual R = dPi/dU (9, n_nodes) of every state."""
        jobs, owner = [], []
        for i, st in enumerate(states):
            for c in self._chunks(st.mesh.n_elems, self.processes):
                jobs.append((st.mesh, st.U, st.Un, st.mask, st.tau, st.material, c))
                owner.append(i)
        parts = self.pool.map(_residual_chunk, jobs, chunksize=1)
        out = [np.zeros_like(st.U) for st in states]
        for i, r in zip(owner, parts):
            out[i] += r
        return out

    def rows_Kx_plus_R(self, state, x: np.ndarray, elements, nodes) -> np.ndarray:
        """(K x + R)[:, nodes] from the contributions of ``elements`` alone:
        the full rows at nodes all of whose adjacent elements are listed."""
        elements = np.asarray(elements)
        jobs = [(state.mesh, state.U, state.Un, state.mask, state.tau, state.material, x, c, nodes)
                for c in np.array_split(elements, self.processes) if c.size]
        rows = sum(self.pool.map(_rows_chunk, jobs, chunksize=1))
        D = state.mask[:, nodes].astype(bool)
        rows[D] = x[:, nodes][D]
        return rows
