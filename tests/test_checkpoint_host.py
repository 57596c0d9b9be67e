"""Checkpoint files are checked before anything is restored (no GPU needed)."""
import numpy as np
import pytest


class _Cloth:
    V, T = 10, 12


def test_load_rejects_other_mesh_and_format(tmp_path):
    from paper_2008_00409_gb300 import checkpoint
    p = tmp_path / "c.npz"
    np.savez(p, format=np.int64(checkpoint.FORMAT), V=np.int64(11), T=np.int64(12))
    with pytest.raises(ValueError, match="another mesh"):
        checkpoint.load(p, _Cloth())
    np.savez(p, format=np.int64(99), V=np.int64(10), T=np.int64(12))
    with pytest.raises(ValueError, match="format"):
        checkpoint.load(p, _Cloth())
