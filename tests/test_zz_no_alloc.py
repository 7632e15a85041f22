"""The attribution entry point that allocates nothing
(cutqc_attribute_noalloc) agrees with cutqc_attribute on a subcircuit that
needs scratch (both initialised and measured cuts), on two calls in a row.
It serves callers that cannot allocate device memory during the call; its
scratch is a static device array of the library.  Collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_attribution_matches_workspace_version():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc as cq
    from workloads import circuits as C
    from workloads.cutting import search_cut
    from workloads.simulate import simulate_variants
    cut = search_cut(C.aqft(14, 7, max_dist=3), 6, 4, restarts=4)
    subs = [s for s in cut.subcircuits if s.k_in > 0 and s.k_out > 0]
    assert subs, "need a subcircuit with both kinds of cut"
    for s in subs:
        assert cq.cutqc_attribute_workspace_size(s) > 0
        v = torch.from_numpy(simulate_variants(s)).cuda()
        ref = cq.cutqc_attribute(s, v)
        shape = ref.shape
        for _ in range(2):
            out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
            cq.cutqc_attribute_noalloc(s, v, out)
            torch.cuda.synchronize()
            r = ref.cpu().numpy().astype(np.float64)
            g = out.cpu().numpy().astype(np.float64)
            assert np.isfinite(g).all()
            assert np.abs(g - r).max() <= 4e-7 * np.abs(r).max()


def test_noalloc_attribution_rejects_oversized_scratch():
    """A subcircuit whose two-pass scratch exceeds the static array (here its
    2^16 x 4^4 float32 measured-side result, 64 MiB > 32 MiB) is refused with
    CUTQC_EUNSUPPORTED before anything is launched: the output keeps its
    contents."""
    import types
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_05836_gb300 import cutqc as cq
    s = types.SimpleNamespace(w=18, in_local=[0, 1], out_local=[16, 17], in_edge=[0, 1], out_edge=[2, 3],
                              out_qubit=list(range(16)))
    assert cq.cutqc_attribute_workspace_size(s) > 32 << 20
    v = torch.zeros((16, 9, 1 << 18), dtype=torch.float32, device="cuda")
    out = torch.full((1 << 16, 256), 7.0, dtype=torch.float32, device="cuda")
    with pytest.raises(cq.CutqcError) as e:
        cq.cutqc_attribute_noalloc(s, v, out)
    assert e.value.code == cq.EUNSUPPORTED
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
