"""The e^x - 1 of the Beeler-Reuter kernels (the Rush-Larsen factor 1 - A =
-(e^{-(alpha+beta) dt} - 1) and the two removable singularities of the rates),
written from the Taylor series of e^x - 1 about 0 near 0 and from e^x - 1
elsewhere, against CUDA's expm1f: within 5e-6 relative over the arguments the
model meets (the bound that follows from the series' first omitted term and
the fast exponential's error on e^x - 1, |e^x - 1| >= 0.22 where it is used)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_expm1_matches_cuda_expm1f():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    xs = np.concatenate([np.linspace(-20.0, 20.0, 400001), np.linspace(-0.3, 0.3, 200001),
                         np.array([0.0, 1e-30, -1e-30, 1e-7, -1e-7, 0.25, -0.25, np.nextafter(0.25, 0)])])
    x = torch.from_numpy(xs.astype(np.float32)).cuda()
    y = torch.empty_like(x)
    ref = torch.empty_like(x)
    bbx.bbx_debug_expm1(x, y, ref)
    y, ref = y.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
    rel = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-38)
    assert rel.max() <= 5e-6, (rel.max(), xs[rel.argmax()])
    assert y[np.nonzero(xs == 0.0)[0][0]] == 0.0
