"""Checkpoint round trip (no GPU)."""
import numpy as np

from paper_2011_08802_gb300 import checkpoint, inputs


def test_checkpoint_round_trip(tmp_path):
    st = inputs.config_indentation(6, seed=3, step=4)
    path = str(tmp_path / "ck.npz")
    checkpoint.save(path, st.U, st.Un, st.mask, st.tau, 4, st.material, st.mesh)
    r = checkpoint.load(path)
    assert np.array_equal(r["U"], st.U) and np.array_equal(r["Un"], st.Un)
    assert np.array_equal(r["mask"], st.mask) and r["tau"] == st.tau and r["load_step"] == 4
    assert r["material"] == st.material
    assert r["mesh"] == (6, 6, 6, st.mesh.Lx, st.mesh.Ly, st.mesh.Lz)
