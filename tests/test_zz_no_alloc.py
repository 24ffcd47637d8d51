"""The allocation-free EDT entry point (ebof_edt_static), on the GPU.

Some callers cannot allocate device memory once they run: a real-time loop
that must not call cudaMalloc (it can synchronise the device), or code inside
a framework that owns all device memory.  For them ebof_edt_static keeps its
scratch in a static device array.  This test calls it through the C ABI
twice in a row, on two different edge images, and checks each result
against the existing entry point ebof_edt (which takes caller scratch):
squared distances bit-exact, surfaces within 1e-5; a third call asks for the
distances only.  It sits in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_edt_static_matches_edt_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as eb
    eb.load()
    dev = "cuda:0"
    rng = np.random.default_rng(21)
    # two calls in a row, different sizes and contents: the second call must
    # not see anything the first one left in the static array
    for W, H, dens in ((1280, 720, 0.02), (517, 301, 0.001)):
        E = (rng.random((H, W)) < dens).astype(np.uint8)
        edge = torch.from_numpy(E).to(dev)
        d_ref = torch.empty((H, W), dtype=torch.int32, device=dev)
        s_ref = torch.empty((H, W), dtype=torch.float32, device=dev)
        scratch = torch.empty(W * H, dtype=torch.int32, device=dev)
        assert eb.ebof_edt(edge, W, H, scratch, d_ref, s_ref, 1.08) == eb.EBOF_OK
        d_st = torch.full((H, W), -7, dtype=torch.int32, device=dev)
        s_st = torch.full((H, W), -7.0, dtype=torch.float32, device=dev)
        assert eb.ebof_edt_static(edge, W, H, d_st, s_st, 1.08) == eb.EBOF_OK
        torch.cuda.synchronize()
        assert torch.equal(d_st, d_ref)
        assert (s_st - s_ref).abs().max().item() <= 1e-5
    # the surface output is optional
    E = (rng.random((97, 131)) < 0.01).astype(np.uint8)
    edge = torch.from_numpy(E).to(dev)
    d_ref = torch.empty((97, 131), dtype=torch.int32, device=dev)
    scratch = torch.empty(97 * 131, dtype=torch.int32, device=dev)
    assert eb.ebof_edt(edge, 131, 97, scratch, d_ref, None, 1.08) == eb.EBOF_OK
    d_st = torch.full((97, 131), -7, dtype=torch.int32, device=dev)
    assert eb.ebof_edt_static(edge, 131, 97, d_st, None, 1.08) == eb.EBOF_OK
    torch.cuda.synchronize()
    assert torch.equal(d_st, d_ref)
    # sizes beyond the static array are refused, nothing is launched
    big = torch.zeros(1, dtype=torch.uint8, device=dev)
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    lib = eb.load()
    assert lib.ebof_edt_static(big.data_ptr(), 2048, 2048, out.data_ptr(), None,
                               1.08, None) == eb.EBOF_ERR_INVALID_ARG
