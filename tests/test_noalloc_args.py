"""The binding of gde_topk_f32_noalloc rejects, before any device work, what the C entry point
cannot see through its plain pointers: host arrays, non-contiguous tensors, wrong dtypes,
outputs shorter than k and tensors on different devices.  Runs on the CPU with stand-in
tensor objects."""
import pytest


class FakeTensor:
    """the attributes of a torch tensor that the binding inspects"""

    def __init__(self, dtype="torch.float32", numel=64, device="cuda:0", cuda=True, contiguous=True):
        self.dtype = dtype
        self.device = device
        self.is_cuda = cuda
        self._numel = numel
        self._contiguous = contiguous

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        raise AssertionError("the binding must not reach the library with bad arguments")


def args(**over):
    a = {"x": FakeTensor(numel=1000), "k": 64, "out_ids": FakeTensor("torch.int32", 64),
         "out_vals": FakeTensor("torch.float32", 64)}
    a.update(over)
    return a


@pytest.mark.parametrize("over, what", [
    ({"x": FakeTensor(cuda=False)}, "CUDA tensor"),
    ({"out_ids": FakeTensor("torch.int32", 64, cuda=False)}, "CUDA tensor"),
    ({"x": FakeTensor(contiguous=False)}, "contiguous"),
    ({"x": FakeTensor("torch.float64", 1000)}, "float32"),
    ({"out_vals": FakeTensor("torch.float16", 64)}, "float32"),
    ({"out_ids": FakeTensor("torch.int64", 64)}, "int32"),
    ({"out_ids": FakeTensor("torch.int32", 63)}, "at least k"),
    ({"out_vals": FakeTensor("torch.float32", 8)}, "at least k"),
    ({"out_vals": FakeTensor("torch.float32", 64, device="cuda:1")}, "one device"),
    ({"x": FakeTensor(numel=1000, device="cuda:1")}, "one device"),
])
def test_topk_noalloc_rejects(over, what):
    import paper_2410_21634_gb300 as gde
    a = args(**over)
    with pytest.raises(ValueError) as e:
        gde.topk_noalloc(a["x"], a["k"], a["out_ids"], a["out_vals"])
    assert what in str(e.value)


def test_topk_noalloc_accepts_valid_arguments():
    import paper_2410_21634_gb300 as gde
    a = args()
    gde._check_topk_noalloc_args(a["x"], a["k"], a["out_ids"], a["out_vals"])
