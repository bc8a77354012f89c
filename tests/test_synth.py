"""The seeded input generators (host side; no GPU)."""
import numpy as np
import torch

from paper_1511_00088_gb300 import synth


def test_device_link_generator_matches_numpy_recipe():
    """random_links_device (torch matrix_exp, same normals) equals random_links
    (numpy eigendecomposition) to rounding, chunk boundary included."""
    L = (4, 4, 4, 8)
    old = synth._CHUNK
    synth._CHUNK = 1000  # several chunks, one boundary inside a direction
    try:
        U = synth.random_links(L, 0.4, 5)
        Ud = synth.random_links_device(L, 0.4, 5, device="cpu").numpy()
    finally:
        synth._CHUNK = old
    assert np.abs(U - Ud).max() < 1e-13
    # SU(3) to rounding
    I = np.eye(3)
    assert np.abs(np.einsum("...ji,...jk->...ik", Ud.conj(), Ud) - I).max() < 1e-13
    assert np.abs(np.linalg.det(Ud) - 1).max() < 1e-13
    assert torch.is_tensor(synth.random_links_device(L, 0.0, 5, device="cpu"))
