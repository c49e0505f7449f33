"""The binding's checks of what the library cannot see behind a pointer
(device, contiguity, element width and kind, shape, sizes), without a GPU.

Device tensors are stood in for by objects with the few attributes the
checks read. The engine under test has no context: a call whose arguments
pass the checks reaches the C boundary, which refuses the null context
(CC_ERR_INVALID_ARG) before any CUDA call. Entry points without a context
(the network's kernels, the static entry) are only driven into their
refusals, so that no kernel is ever launched on a stand-in pointer.
"""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import paper_1607_06156_gb300 as cc


class Dev:
    """A stand-in for a CUDA tensor."""

    def __init__(self, shape, dtype=torch.int32, cuda=True, index=0, contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = cuda
        self.device = SimpleNamespace(type="cuda" if cuda else "cpu", index=index if cuda else None)
        self._contiguous = contiguous

    def is_contiguous(self):
        return self._contiguous

    def element_size(self):
        return self.dtype.itemsize

    def numel(self):
        return int(np.prod(self.shape)) if self.shape else 1

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return 0x10000


def _engine(id_bytes=4):
    eng = object.__new__(cc.Engine)
    eng._opt = cc.default_options()
    eng._opt.id_bytes = id_bytes
    eng.device = 0
    eng._h = None
    return eng


def _reaches_the_boundary(call):
    with pytest.raises(cc.CCError) as ei:
        call()
    assert ei.value.status == 1  # the null context, refused by the library


@pytest.mark.parametrize("method", ["labels", "labels_tuple_sv"])
def test_labels_checks(method):
    eng = _engine(4)
    f = getattr(eng, method)
    e, out = Dev((100, 2)), Dev((50,))
    _reaches_the_boundary(lambda: f(e, 50, out=out, stream=0))
    _reaches_the_boundary(lambda: f(Dev((0, 2)), 50, out=out, stream=0))
    bad = [
        (Dev((100, 2), cuda=False), out, "CUDA"),
        (Dev((100, 2), index=1), out, "engine"),
        (Dev((100, 2), contiguous=False), out, "contiguous"),
        (Dev((100, 2), torch.int64), out, "4-byte"),
        (Dev((100, 2), torch.float32), out, "integer"),
        (Dev((200,)), out, "shape"),
        (Dev((100, 3)), out, "shape"),
        (e, Dev((49,)), "50 are needed"),
        (e, Dev((50,), torch.int64), "4-byte"),
        (e, Dev((50,), cuda=False), "CUDA"),
    ]
    for edges, o, msg in bad:
        with pytest.raises(ValueError, match=msg):
            f(edges, 50, out=o, stream=0)
    eng8 = _engine(8)
    _reaches_the_boundary(lambda: getattr(eng8, method)(Dev((10, 2), torch.int64), 5,
                                                       out=Dev((5,), torch.int64), stream=0))
    with pytest.raises(ValueError, match="8-byte"):
        getattr(eng8, method)(Dev((10, 2), torch.complex64), 5, out=Dev((5,), torch.int64), stream=0)


def test_labels_host_checks():
    eng = _engine(4)
    e = torch.zeros((10, 2), dtype=torch.int32)
    _reaches_the_boundary(lambda: eng.labels_host(e, 5, stream=0))
    for edges, msg in ((torch.zeros((10, 2), dtype=torch.int64), "4-byte"),
                       (torch.zeros((10, 2), dtype=torch.float32), "4-byte"),
                       (torch.zeros(20, dtype=torch.int32), "shape"),
                       (torch.zeros((2, 10), dtype=torch.int32).t(), "contiguous")):
        with pytest.raises(ValueError, match=msg):
            eng.labels_host(edges, 5, stream=0)
    with pytest.raises(ValueError, match="out"):
        eng.labels_host(e, 5, out=torch.zeros(4, dtype=torch.int32), stream=0)


def test_batched_checks():
    eng = _engine(4)
    e = Dev((30, 2))
    eo, vo = np.array([0, 10, 30]), np.array([0, 100, 150])
    for edges, eoff, voff, msg in (
            (Dev((30, 2), torch.int64), eo, vo, "4-byte"),
            (e, np.array([0, 10, 31]), vo, "the edges hold 30"),
            (e, eo, np.array([0, 100]), "G \\+ 1"),
            (e, np.zeros((2, 2)), np.zeros((2, 2)), "1-D"),
            (e, eo, vo, "out holds")):
        with pytest.raises(ValueError, match=msg):
            eng.labels_batched(edges, torch.as_tensor(eoff), torch.as_tensor(voff), out=Dev((149,)), stream=0)
    with pytest.raises(ValueError, match="the edges hold 30"):
        eng.ks_statistic_batched(e, np.array([0, 40]), np.array([0, 5]), stream=0)
    _reaches_the_boundary(lambda: eng.labels_batched_dev(e, Dev((3,), torch.int64), Dev((3,), torch.int64), 30, 150,
                                                         Dev((150,)), stream=0))
    for eod, vod, m_tot, n_tot, o, msg in (
            (Dev((2,), torch.int64), Dev((3,), torch.int64), 30, 150, Dev((150,)), "G \\+ 1"),
            (Dev((3,)), Dev((3,), torch.int64), 30, 150, Dev((150,)), "8-byte"),
            (Dev((3,), torch.int64), Dev((3,), torch.int64), 31, 150, Dev((150,)), "within the 30 pairs"),
            (Dev((3,), torch.int64), Dev((3,), torch.int64), 30, -1, Dev((150,)), "n_total"),
            (Dev((3,), torch.int64), Dev((3,), torch.int64), 30, 150, Dev((100,)), "150 are needed")):
        with pytest.raises(ValueError, match=msg):
            eng.labels_batched_dev(e, eod, vod, m_tot, n_tot, o, stream=0)


def test_degree_ks_and_feature_checks():
    eng = _engine(8)
    e = Dev((10, 2), torch.int64)
    _reaches_the_boundary(lambda: eng.ks_statistic(Dev((7,), torch.int64), stream=0))
    with pytest.raises(ValueError, match="8-byte"):
        eng.ks_statistic(Dev((7,), torch.int32), stream=0)
    with pytest.raises(ValueError, match="1 are needed"):
        eng.ks_statistic(Dev((0,), torch.int64), stream=0)
    with pytest.raises(ValueError, match="8-byte"):
        eng.degree_distribution(Dev((10, 2)), 5, stream=0)
    with pytest.raises(ValueError, match="shape"):
        eng.route_features(Dev((10, 4), torch.int64), 5, stream=0)
    with pytest.raises(ValueError, match="CUDA"):
        eng.route_features(Dev((10, 2), torch.int64, cuda=False), 5, stream=0)
    del e


def test_network_and_static_entry_refusals():
    P = Dev((cc.MLP_PARAMS,), torch.float32)
    X = Dev((8, cc.MLP_IN), torch.float32)
    act = Dev((8 * (2 * cc.MLP_HIDDEN + cc.MLP_OUT),), torch.float32)
    with pytest.raises(ValueError, match="params holds"):
        cc.mlp_forward(Dev((cc.MLP_PARAMS - 1,), torch.float32), X, act, stream=0)
    with pytest.raises(ValueError, match="shape"):
        cc.mlp_forward(P, Dev((8, cc.MLP_IN + 1), torch.float32), act, stream=0)
    with pytest.raises(ValueError, match="floating-point"):
        cc.mlp_forward(P, Dev((8, cc.MLP_IN), torch.int32), act, stream=0)
    with pytest.raises(ValueError, match="act holds"):
        cc.mlp_forward(P, X, Dev((act.numel() - 1,), torch.float32), stream=0)
    f = lambda k: Dev((k,), torch.float32)
    good = dict(y=Dev((8,)), t=f(8), w=f(8), act=act, grad=f(cc.MLP_PARAMS), scratch=f(8 * (3 + 2 * cc.MLP_HIDDEN)),
                loss=f(1))
    for k, v in (("y", Dev((8,), torch.float32)), ("t", f(7)), ("scratch", f(8 * (3 + 2 * cc.MLP_HIDDEN) - 1)),
                 ("grad", f(10)), ("loss", f(0))):
        kw = dict(good, **{k: v})
        with pytest.raises(ValueError, match=k):
            cc.mlp_backward(P, X, kw["y"], kw["t"], kw["w"], 0.1, kw["act"], kw["grad"], kw["scratch"], kw["loss"],
                            stream=0)
    with pytest.raises(ValueError, match="grad holds"):
        cc.mlp_adam(P, f(10), P, P, 1e-3, 1, stream=0)
    with pytest.raises(ValueError, match="v must"):
        cc.mlp_adam(P, P, P, Dev((cc.MLP_PARAMS,), torch.float32, contiguous=False), 1e-3, 1, stream=0)
    with pytest.raises(ValueError, match="out holds"):
        cc.labels_static(Dev((10, 2)), 5, out=Dev((4,)), stream=0)
    with pytest.raises(ValueError, match="integer"):
        cc.labels_static(Dev((10, 2), torch.float32), 5, out=Dev((5,)), stream=0)
