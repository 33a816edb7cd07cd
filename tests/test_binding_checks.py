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


def _static_args(n_mod=4, n_hits=5, cap=8):
    return dict(modules=FakeCuda((n_mod * lst.LST_MODULE_BYTES,), "torch.uint8"),
                x=FakeCuda((n_hits,)), y=FakeCuda((n_hits,)), z=FakeCuda((n_hits,)),
                module=FakeCuda((n_hits,), "torch.int32"), side=FakeCuda((n_hits,), "torch.uint8"),
                md_lower=FakeCuda((cap,), "torch.int32"), md_upper=FakeCuda((cap,), "torch.int32"),
                md_module=FakeCuda((cap,), "torch.int32"), md_dphi=FakeCuda((cap,)), md_dlong=FakeCuda((cap,)),
                md_count=FakeCuda((1,), "torch.int32"), md_dropped=FakeCuda((1,), "torch.int32"))


@pytest.mark.parametrize("key,bad,match", [
    ("modules", FakeCuda((4 * 20 - 1,), "torch.uint8"), "needed"),
    ("modules", FakeCuda((80,), "torch.int32"), "dtype"),
    ("x", np.zeros(5, np.float32), "CUDA tensor"),
    ("y", FakeCuda((4,)), "needed"),
    ("z", FakeCuda((5,), contiguous=False), "contiguous"),
    ("module", FakeCuda((5,), "torch.int64"), "dtype"),
    ("side", FakeCuda((5,), "torch.bool"), "dtype"),
    ("md_lower", FakeCuda((7,), "torch.int32"), "needed"),
    ("md_upper", FakeCuda((8,)), "dtype"),
    ("md_module", FakeCuda((7,), "torch.int32"), "needed"),
    ("md_dphi", FakeCuda((7,)), "needed"),
    ("md_dlong", FakeCuda((8,), "torch.float64"), "dtype"),
    ("md_count", FakeCuda((0,), "torch.int32"), "needed"),
    ("md_dropped", FakeCuda((1,), "torch.float32"), "dtype"),
])
def test_static_builder_refuses_bad_arrays_before_calling_the_library(key, bad, match):
    """Every array of the allocation-free MD builder is read or written by pointer on the device: a wrong dtype,
    a strided view or an array shorter than n_mod rows / n_hits / md_capacity is refused on the host."""
    assert lst.LST_MODULE_BYTES == 20
    a = _static_args()
    a[key] = bad
    with pytest.raises(LstError, match=match):
        lst.build_mini_doublets_static(None, a.pop("modules"), 4, a.pop("x"), a.pop("y"), a.pop("z"),
                                       a.pop("module"), a.pop("side"), 5, 8, **a)


def test_static_builder_refuses_negative_sizes():
    a = _static_args()
    for n_mod, n_hits, cap in ((0, 5, 8), (4, -1, 8), (4, 5, -1)):
        b = dict(a)
        with pytest.raises(LstError, match="required"):
            lst.build_mini_doublets_static(None, b.pop("modules"), n_mod, b.pop("x"), b.pop("y"), b.pop("z"),
                                           b.pop("module"), b.pop("side"), n_hits, cap, **b)
