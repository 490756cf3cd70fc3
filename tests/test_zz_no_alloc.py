"""The allocation-free MRG32K3A entry point against the ordinary one.

prand_mrg32k3a_generate_u32_noalloc serves callers that cannot allocate device
memory (all memory owned by their own allocator or a fixed budget, or code
running where an allocation would synchronise the device).  It keeps its
scratch in a fixed array inside the library.  Here its output and the states it
leaves behind must equal prand_generate_u32 on a handle holding the same
streams, bit for bit, on two calls in a row.  The file sorts last so that a
failure here never hides another test's result.
"""
import numpy as np
import pytest

import paper_1307_5869_gb300 as P

pytestmark = pytest.mark.gpu


def _payload(blob: bytes, n_streams: int) -> np.ndarray:
    words = 6 * n_streams
    return np.frombuffer(blob[len(blob) - 4 * words:], dtype=np.uint32).copy()


@pytest.mark.parametrize("n_streams,n_per", [(3, 50_000), (4096, 1000), (65536, 64)])
def test_noalloc_matches_handle_on_two_calls(n_streams, n_per):
    import torch
    P.load(build_if_missing=True)
    g = P.Generator("MRG32K3A", 2024, 17, n_streams)
    st = torch.from_numpy(_payload(g.get_state(), n_streams).view(np.int32)).cuda()
    out = torch.empty(n_streams * n_per, dtype=torch.int32, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        ref = g.generate(n_per, "u32").reshape(-1)
        P.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), n_streams, out.data_ptr(), n_per, sp)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), f"call {call}: outputs differ"
        assert np.array_equal(st.cpu().numpy().view(np.uint32), _payload(g.get_state(), n_streams)), \
            f"call {call}: states differ"
    g.close()


def test_noalloc_rejects_too_many_streams():
    import torch
    L = P.load(build_if_missing=True)
    st = torch.zeros(6, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    assert L.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), 65537, out.data_ptr(), 1, None) == 1
    assert L.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), 0, out.data_ptr(), 1, None) == 1


def test_noalloc_second_call_on_another_stream():
    # the set-up happens once per device; a later call on a different stream
    # (here a fresh torch stream) runs with it and still equals the handle path
    import torch
    P.load(build_if_missing=True)
    n_streams, n_per = 1000, 4096
    g = P.Generator("MRG32K3A", 77, 5, n_streams)
    st = torch.from_numpy(_payload(g.get_state(), n_streams).view(np.int32)).cuda()
    out = torch.empty(n_streams * n_per, dtype=torch.int32, device="cuda")
    first = torch.cuda.current_stream()
    P.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), n_streams, out.data_ptr(), n_per, first.cuda_stream)
    ref = g.generate(n_per, "u32").reshape(-1)
    torch.cuda.synchronize()
    assert torch.equal(out, ref), "call on the current stream differs"
    other = torch.cuda.Stream()
    with torch.cuda.stream(other):
        P.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), n_streams, out.data_ptr(), n_per, other.cuda_stream)
    other.synchronize()
    ref = g.generate(n_per, "u32").reshape(-1)
    torch.cuda.synchronize()
    assert torch.equal(out, ref), "call on another stream differs"
    assert np.array_equal(st.cpu().numpy().view(np.uint32), _payload(g.get_state(), n_streams))
    g.close()


def test_noalloc_zero_outputs_leaves_states_unchanged():
    import torch
    P.load(build_if_missing=True)
    n_streams = 64
    g = P.Generator("MRG32K3A", 5, 0, n_streams)
    before = _payload(g.get_state(), n_streams)
    st = torch.from_numpy(before.view(np.int32)).cuda()
    out = torch.full((4,), -1, dtype=torch.int32, device="cuda")
    P.prand_mrg32k3a_generate_u32_noalloc(st.data_ptr(), n_streams, out.data_ptr(), 0,
                                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.array_equal(st.cpu().numpy().view(np.uint32), before)
    assert (out.cpu() == -1).all(), "a fill of zero outputs wrote to the output"
    g.close()
