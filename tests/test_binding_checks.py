"""Input checks of the Python binding (CPU): arrays the library would read on
the device, or read past their end, are refused before any call is made."""
import numpy as np
import pytest
import torch

from paper_2209_13711_gb300 import LstError, lst


class FakeCuda:
    """Stands in for a CUDA tensor (never reaches the library)."""

    def __init__(self, shape, dtype="torch.float32", contiguous=True):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = True
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return int(np.prod(self.shape))

    def data_ptr(self):
        return 0


def _host(n_hits=5, n_seeds=2):
    return dict(x=np.zeros(n_hits, np.float32), y=np.zeros(n_hits, np.float32), z=np.zeros(n_hits, np.float32),
                module=np.zeros(n_hits, np.int32), side=np.zeros(n_hits, np.uint8),
                seeds=np.zeros((n_seeds, 3, 3), np.float32))


def test_host_inputs_numpy_and_cpu_tensors():
    assert lst._input_kind(_host(), 5, 2) is False
    t = {k: torch.from_numpy(v) for k, v in _host().items()}
    assert lst._input_kind(t, 5, 2) is False
    assert lst._input_kind(lst.pack_events([]), 0, 0) is False


def test_device_inputs():
    d = dict(x=FakeCuda((5,)), y=FakeCuda((5,)), z=FakeCuda((5,)), module=FakeCuda((5,), "torch.int32"),
             side=FakeCuda((5,), "torch.uint8"), seeds=FakeCuda((2, 9)))
    assert lst._input_kind(d, 5, 2) is True
    d["seeds"] = np.zeros(18, np.float32)
    with pytest.raises(LstError, match="mix"):
        lst._input_kind(d, 5, 2)


@pytest.mark.parametrize("key,bad", [("module", np.zeros(5, np.int64)), ("side", np.zeros(5, bool)),
                                     ("x", np.zeros(5, np.float64)), ("z", np.zeros(4, np.float32)),
                                     ("y", np.zeros(10, np.float32)[::2]), ("seeds", np.zeros(17, np.float32))])
def test_bad_host_inputs(key, bad):
    d = _host()
    d[key] = bad
    with pytest.raises(LstError):
        lst._input_kind(d, 5, 2)


def test_context_refuses_before_calling_the_library():
    ctx = object.__new__(lst.Context)          # no device: the checks come first
    b = lst.pack_events([])
    b["hit_off"] = np.array([0, 3], np.int32)  # claims 3 hits, arrays hold 0
    with pytest.raises(LstError, match="needed"):
        ctx.run_packed(b)
    evs = [_host(), {k: torch.from_numpy(v) for k, v in _host().items()}]
    evs[1]["x"] = FakeCuda((5,))
    with pytest.raises(LstError, match="mix"):
        ctx.run_events(evs)


def test_network_arrays_must_be_device_float32_of_the_right_shape():
    m = object.__new__(lst.Mlp)
    f, s = FakeCuda((7, 48)), FakeCuda((7,))
    assert lst._device_array(f, "features", "float32", (7, 48)) is not None
    with pytest.raises(LstError, match="CUDA tensor"):
        m.forward(np.zeros((7, 48), np.float32), s)
    with pytest.raises(LstError, match="shape"):
        m.forward(FakeCuda((7, 38)), s)
    with pytest.raises(LstError, match="dtype"):
        m.gradient(f, FakeCuda((7,), "torch.float64"))
    with pytest.raises(LstError, match="contiguous"):
        m.train_step(FakeCuda((7, 48), contiguous=False), s)
