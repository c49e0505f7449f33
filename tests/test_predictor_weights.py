"""The shipped route-predictor weights file (CPU only)."""
import numpy as np


def test_committed_route_predictor_weights_load():
    """The shipped weights file parses, its CRC-32 matches and it holds one
    parameter per network weight."""
    from paper_1607_06156_gb300 import MLP_PARAMS
    from paper_1607_06156_gb300.train_predictor import default_weights_path, load_params

    p, n_train = load_params(default_weights_path())
    assert p.size == MLP_PARAMS and n_train >= 20000
    assert np.isfinite(p).all()
