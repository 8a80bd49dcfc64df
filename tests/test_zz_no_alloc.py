"""bbx_total_noalloc: the tissue sum for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library).  Checked
against bbx_total, the allocating entry point, on two calls in a row.  This
file is collected last so that a failure here does not hide the others."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_total_matches_bbx_total_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_06015_gb300 import bbx
    from paper_1605_06015_gb300 import workloads as wl

    nx, ny, nz = 150, 70, 20
    mask, fib = wl.random_geometry(nx, ny, nz, seed=3, tissue_frac=0.7)
    G = bbx.Grid(nx, ny, nz, 0.3, mask)
    G.set_fibres(fib, 1.0, 0.25)
    G.set_ionic_model(bbx.BBX_BARKLEY)
    G.write_state(0, np.random.default_rng(4).random((nz, ny, nx)).astype(np.float32))  # u in [0, 1)
    px = G.get_info()["px"]
    # the caller owns the mask and the output (pitched like the field)
    dmask = torch.zeros((nz, ny, px), dtype=torch.uint8, device="cuda")
    dmask[:, :, :nx] = torch.from_numpy(mask)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        ref = G.total(0)
        bbx.bbx_total_noalloc(G.state_device_ptr(0), dmask.data_ptr(), nx, ny, nz, px, out.data_ptr(), stream)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=1e-12), call
        G.step(0.005, 3)  # different data for the second call
    # whole field, no mask
    bbx.bbx_total_noalloc(G.state_device_ptr(0), None, nx, ny, nz, px, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(float(np.sum(G.read_state(0).astype(np.float64))), rel=1e-12)
    # few long rows (fewer rows than SMs): each block walks whole rows
    u2 = torch.rand((1, 3, 70001), dtype=torch.float32, device="cuda")
    bbx.bbx_total_noalloc(u2.data_ptr(), None, 70001, 3, 1, 70001, out.data_ptr(), stream)
    torch.cuda.synchronize()
    assert out.item() == pytest.approx(float(u2.double().sum().item()), rel=1e-12)
    # a field beyond the fixed scratch (2^28 nodes) is refused before any launch
    with pytest.raises(bbx.BbxError) as e:
        bbx.bbx_total_noalloc(G.state_device_ptr(0), None, 1 << 15, 1 << 14, 2, 1 << 15, out.data_ptr(), stream)
    assert e.value.code == bbx.BBX_ERR_ARG
