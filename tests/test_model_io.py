"""The compact model layout (Sec. IV): size formula pinned by the paper's example,
and a lossless round trip of binary32 models (no GPU)."""
import os

import numpy as np

from paper_2307_00071_gb300 import model_io, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "model_size.txt")


def test_model_size_matches_the_papers_example():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    for d, m, nbytes in rows:
        assert model_io.model_bytes(int(m), int(d)) == int(nbytes)
    assert model_io.floats_per_component(3) == 10 and model_io.floats_per_component(4) == 15


def test_pack_unpack_round_trip():
    for cl, d in ((synth.gmm_cloud4(100, 7, seed=1), 4), (synth.gmm_cloud(100, 5, seed=2), 3)):
        w, m, c = (np.asarray(a, np.float32) for a in (cl.weights, cl.means, cl.covs))
        c = 0.5 * (c + np.transpose(c, (0, 2, 1)))
        data = model_io.pack_model(w, m, c)
        assert len(data) == model_io.model_bytes(len(w), d)
        w2, m2, c2 = model_io.unpack_model(data, d)
        np.testing.assert_array_equal(w2, w)
        np.testing.assert_array_equal(m2, m)
        np.testing.assert_array_equal(c2, c)
