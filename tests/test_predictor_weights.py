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


def test_weights_file_round_trip_and_corruption(tmp_path):
    """save_params / load_params keep every bit; a flipped byte, a wrong magic
    or another version is refused."""
    import struct
    import zlib

    import pytest

    from paper_1607_06156_gb300.train_predictor import MAGIC, load_params, save_params

    p = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    path = str(tmp_path / "w.bin")
    save_params(path, p, 1234)
    q, n_train = load_params(path)
    assert n_train == 1234 and q.dtype == np.float32 and np.array_equal(q.view(np.uint32), p.view(np.uint32))
    raw = bytearray(open(path, "rb").read())
    bad = bytearray(raw)
    bad[100] ^= 0x01
    open(path, "wb").write(bytes(bad))
    with pytest.raises(ValueError):
        load_params(path)
    body = b"XXXX" + bytes(raw[4:-4])
    open(path, "wb").write(body + struct.pack("<I", zlib.crc32(body) & 0xffffffff))
    with pytest.raises(ValueError):
        load_params(path)
    body = MAGIC + struct.pack("<I", 2) + bytes(raw[8:-4])
    open(path, "wb").write(body + struct.pack("<I", zlib.crc32(body) & 0xffffffff))
    with pytest.raises(ValueError):
        load_params(path)


def test_training_targets_from_route_timings():
    """Column 0 is SV only, columns 1.. are BFS with each cutoff: the target
    is BFS iff its best cutoff beats SV, with the log of that cutoff (BFS to
    completion stands for 64 levels) weighted only where BFS won."""
    from paper_1607_06156_gb300.train_predictor import CUTOFFS, NO_CUTOFF_LEVELS, targets

    assert len(CUTOFFS) == 5
    T = np.array([[1.0, 2.0, 3.0, 4.0, 5.0, 6.0],    # SV fastest
                  [9.0, 5.0, 4.0, 3.0, 8.0, 9.0],    # BFS with cutoff 8
                  [9.0, 5.0, 5.0, 5.0, 5.0, 1.0],    # BFS to completion
                  [2.0, 3.0, 2.5, 2.0, 2.0, 2.0]])   # a tie with SV goes to SV
    y, t, w = targets(T)
    assert y.tolist() == [0, 1, 1, 0]
    assert np.allclose(t, np.log([2.0, 8.0, NO_CUTOFF_LEVELS, 8.0]))
    assert w.tolist() == [0.0, 1.0, 1.0, 0.0]


def test_parameter_layout_and_constant_network():
    """The flat layout holds W1, b1, W2, b2, W3, b3 (He-uniform weights, zero
    biases); the constant network picks its route and cutoff on any input
    (evaluated with the fp64 oracle network)."""
    from oracle import mlp
    from paper_1607_06156_gb300 import MLP_HIDDEN, MLP_IN, MLP_OUT, MLP_PARAMS
    from paper_1607_06156_gb300.train_predictor import constant_params, init_params

    p = init_params(3)
    assert p.size == MLP_PARAMS and p.dtype == np.float32
    o = 0
    for fo, fi in ((MLP_HIDDEN, MLP_IN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_OUT, MLP_HIDDEN)):
        W, b = p[o:o + fo * fi], p[o + fo * fi:o + fo * fi + fo]
        lim = np.sqrt(6.0 / fi)
        assert np.abs(W).max() <= lim and np.abs(W).max() > 0.9 * lim and not b.any()
        o += fo * fi + fo
    assert o == MLP_PARAMS

    def unflat(f):
        out, o = {}, 0
        for k, shp in (("W1", (MLP_HIDDEN, MLP_IN)), ("b1", (MLP_HIDDEN,)), ("W2", (MLP_HIDDEN, MLP_HIDDEN)),
                       ("b2", (MLP_HIDDEN,)), ("W3", (MLP_OUT, MLP_HIDDEN)), ("b3", (MLP_OUT,))):
            c = int(np.prod(shp))
            out[k] = f[o:o + c].reshape(shp).astype(np.float64)
            o += c
        return out

    X = np.random.default_rng(1).standard_normal((7, MLP_IN))
    for route, cutoff, levels in ((0, 4, 4.0), (1, 8, 8.0), (1, 0, 64.0)):
        out = mlp.forward(unflat(constant_params(route, cutoff)), X)["o"]
        assert ((out[:, 1] > out[:, 0]).astype(int) == route).all()
        assert np.allclose(out[:, 2], np.log(levels))
