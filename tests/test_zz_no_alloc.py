"""The allocation-free forward transform (grouped_trafo_noalloc) agrees with the
plan-based grouped_trafo.

grouped_trafo_noalloc exists for callers that cannot allocate device memory
when they need a transform (their device memory is reserved by their own pool,
or they run inside a callback or a latency-critical loop where cudaMalloc and
cudaFree are not allowed); its working memory is a static device array inside
the library.  This file is named so that pytest collects it after every other
test file: it must pass in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from oracle import ndft
from paper_2010_10199_gb300 import inputs

from gpu_util import cplx_dev, f32_nodes, host, rel_l2, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5   # the FP32 transform tolerance used by the other GPU tests


def test_noalloc_matches_plan_path_twice_in_a_row():
    import torch
    from paper_2010_10199_gb300 import build, gft
    build.build()
    gft.load()
    w = inputs.c2_scale(M=20000)
    terms, bw = w["terms"], w["bandwidths"]
    x = to_dev(w["x"], torch.float32)
    P = gft.Plan(x, terms, bw)
    stream = torch.cuda.current_stream()
    for seed in (1, 2):   # two calls in a row, different coefficients
        fhat = cplx_dev(inputs.decaying_coefficients(seed, terms, bw))
        ref = host(P.trafo(fhat))
        f = torch.full((w["M"],), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
        gft.grouped_trafo_noalloc(20, w["M"], x.data_ptr(), terms, bw, fhat.data_ptr(), f.data_ptr(),
                                  stream.cuda_stream)
        torch.cuda.synchronize()
        out = host(f)
        assert np.all(np.isfinite(out))
        assert rel_l2(out, ref) <= TOL


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2010_10199_gb300 import gft
    gft.load()
    terms = inputs.terms_up_to(20, 2)
    bw = inputs.bandwidths_by_order(terms, {1: 64, 2: 32})
    M = 1_000_000   # nodes alone need 80 MB, beyond the 32 MiB array
    n = inputs.coeff_count(terms, bw)
    x = torch.zeros((20, M), dtype=torch.float32, device="cuda")      # real buffers of the stated sizes
    fhat = torch.zeros(n, dtype=torch.complex64, device="cuda")
    f = torch.zeros(M, dtype=torch.complex64, device="cuda")
    with pytest.raises(gft.AnovaError) as e:
        gft.grouped_trafo_noalloc(20, M, x.data_ptr(), terms, bw, fhat.data_ptr(), f.data_ptr(), 0)
    assert e.value.status == -2
    torch.cuda.synchronize()
    assert float(f.abs().max()) == 0.0   # nothing was written


def test_noalloc_third_order_terms_match_oracle_and_plan_path():
    """Third-order terms (grids without halos, indices modulo n, the
    point-major gather) through the allocation-free call, against the FP64
    oracle and against grouped_trafo."""
    import torch
    from paper_2010_10199_gb300 import build, gft
    build.build()
    gft.load()
    d, M = 4, 5000
    x = inputs.uniform_points(31, d, M)
    terms = inputs.terms_up_to(d, 3)
    bw = inputs.bandwidths_by_order(terms, {1: 20, 2: 12, 3: 10})
    fh = inputs.decaying_coefficients(4, terms, bw)
    xd = to_dev(x, torch.float32)
    fhat = cplx_dev(fh)
    f = torch.full((M,), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    gft.grouped_trafo_noalloc(d, M, xd.data_ptr(), terms, bw, fhat.data_ptr(), f.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out = host(f)
    ref = ndft.trafo(f32_nodes(x), terms, bw, fh)
    assert rel_l2(out, ref) <= TOL
    P = gft.Plan(xd, terms, bw)
    assert rel_l2(out, host(P.trafo(fhat))) <= TOL


def test_noalloc_refuses_a_capturing_stream():
    """While the stream is capturing a CUDA graph the call returns
    ANOVA_ERR_UNSUPPORTED and enqueues nothing (its table uploads read host
    staging memory that the next call overwrites)."""
    import torch
    from paper_2010_10199_gb300 import gft
    gft.load()
    w = inputs.c1_small()
    terms, bw, M = w["terms"], w["bandwidths"], w["M"]
    x = to_dev(w["x"], torch.float32)
    fhat = cplx_dev(inputs.decaying_coefficients(2, terms, bw))
    f = torch.zeros(M, dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            gft.grouped_trafo_noalloc(6, M, x.data_ptr(), terms, bw, fhat.data_ptr(), f.data_ptr(), s.cuda_stream)
        except gft.AnovaError as e:
            status = e.status
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert status == -2
    assert float(f.abs().max()) == 0.0
