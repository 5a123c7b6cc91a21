"""The Python binding refuses buffers of the wrong shape, dtype, layout or device before
any pointer reaches the C ABI (which sees raw pointers and sizes only).  CPU only: the
checks run before any CUDA call."""
import numpy as np
import pytest
import torch

from paper_2504_04941_gb300 import inputs as I
from paper_2504_04941_gb300 import kt


class FakeCuda:
    """Stands in for a CUDA tensor: only the attributes the checks read."""

    def __init__(self, shape, dtype="float64", contiguous=True):
        self.shape = tuple(shape)
        self.dtype = f"torch.{dtype}"
        self.is_cuda = True
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def dim(self):
        return len(self.shape)


@pytest.fixture(scope="module")
def net():
    from paper_2504_04941_gb300 import build
    build.build()                     # host-only use of the library (network parsing)
    return kt.Network(I.network(2))


def test_cpu_tensors_are_refused(net):
    wl = I.workload(2, 8)
    y, T = torch.from_numpy(wl.cells.y), torch.from_numpy(wl.cells.T)
    with pytest.raises(ValueError, match="CUDA"):
        kt.integrate(net, y, T, 1e-9, kt.options(wl.tol))
    with pytest.raises(ValueError, match="CUDA"):
        kt.integrate_noalloc(net, y, T, 1e-9, kt.options(wl.tol), dict(y=y, T=T))


def test_cell_buffer_shapes_dtypes_and_layout(net):
    ns = net.ns
    ok = dict(y=FakeCuda((ns, 5)), T=FakeCuda((5,)))
    assert kt._require_cells(net, ok["y"], ok["T"], FakeCuda((5,)), dict(status=FakeCuda((5,), "int32"))) == 5
    bad = [
        (FakeCuda((ns + 1, 5)), FakeCuda((5,)), None, None),              # species count
        (FakeCuda((ns, 4)), FakeCuda((5,)), None, None),                  # cell count
        (FakeCuda((ns, 5), "float32"), FakeCuda((5,)), None, None),       # dtype
        (FakeCuda((ns, 5), contiguous=False), FakeCuda((5,)), None, None),
        (FakeCuda((ns, 5)), FakeCuda((5,)), FakeCuda((4,)), None),        # rho length
        (FakeCuda((ns, 5)), FakeCuda((5,)), None, dict(y=FakeCuda((ns, 6)))),
        (FakeCuda((ns, 5)), FakeCuda((5,)), None, dict(status=FakeCuda((5,), "int64"))),
        (FakeCuda((ns, 5)), FakeCuda((5, 1)), None, None),                # T not 1-D
    ]
    for y, T, rho, outs in bad:
        with pytest.raises(ValueError):
            kt._require_cells(net, y, T, rho, outs)


def test_host_arrays(net):
    kt._require_host(np.zeros((net.ns, 3)), "y", (net.ns, 3), np.float64)
    kt._require_host(None, "rho", (3,), np.float64, optional=True)
    for a in (np.zeros((net.ns, 3), np.float32), np.zeros((3, net.ns)).T, np.zeros((net.ns, 4)), [0.0] * 3):
        with pytest.raises(ValueError):
            kt._require_host(a, "y", (net.ns, 3), np.float64)
    with pytest.raises(ValueError):
        kt._require_host(None, "y", (net.ns, 3), np.float64)
