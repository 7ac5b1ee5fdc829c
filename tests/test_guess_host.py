"""Host-side pieces of the learned initial guess (no GPU): the flat parameter layout that
the library's network reads, and the stored trained weights."""
import os

import numpy as np

from oracle import unet as ounet
from paper_2403_01039_gb300 import capi, guess


def test_initial_weights_use_the_network_layout():
    """guess.init_flat draws the same He-normal values, layer by layer, as the oracle network's
    init_params, in the flat order weights-then-biases per layer: the two must coincide once
    flattened (so a trained vector means the same layers on both sides)."""
    for channels in ((16, 32, 64), (4, 6, 8)):
        flat = guess.init_flat(5, 5, seed=3, channels=channels)
        ref = capi.flatten_params(ounet.init_params(5, 5, seed=3, channels=channels))
        assert flat.dtype == np.float32 and np.array_equal(flat, ref)
        back = capi.unflatten(flat.astype(np.float64), ounet.init_params(5, 5, seed=0, channels=channels))
        assert [w.shape for w, _ in back][-1] == (5, channels[0])


def test_stored_weights_fit_the_layout():
    path = os.path.join(os.path.dirname(capi.__file__), "data", "guess_unet_solute50_128.npz")
    W = np.load(path)
    channels = tuple(int(c) for c in W["channels"])
    assert channels == guess.CHANNELS and int(W["crop"]) == guess.CROP
    n = capi.flatten_params(ounet.init_params(5, 5, seed=0, channels=channels)).size
    assert W["params"].dtype == np.float32 and W["params"].size == n
    assert np.all(np.isfinite(W["params"]))
    hist = np.asarray(W["history"])
    assert hist.size >= 2 and hist[-1] < hist[0]          # the training loss went down
