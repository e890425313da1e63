"""snn_rewire_deepr_noalloc: DEEP R rewiring for callers that cannot allocate device
memory (a serving process with a fixed, pre-reserved memory budget, or a host framework
whose allocator owns every buffer).  It must give exactly what the handle-based
snn_rewire_deepr gives on the same state, call after call, while using only the
library's fixed static scratch.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _plain_copy(d, dev="cuda"):
    """Second set of caller-owned arrays with the same contents as handle `d`, and a
    plain descriptor pointing at them (no handle is created for it)."""
    from paper_2510_19764_gb300 import abi
    arrs = {k: getattr(d, k).clone() for k in ("row_len", "ind", "w", "m", "v", "sign_bits", "conn_bits")}
    desc = abi.RaggedDesc()
    desc.P, desc.Q, desc.C, desc.dtype, desc.no_autapse, desc.reserved = d.P, d.Q, d.C, d.dtype, d.desc.no_autapse, 0
    for k in ("row_len", "ind", "w", "m", "v", "sign_bits", "conn_bits"):
        setattr(desc, k, abi.ptr(arrs[k]))
    desc.grad = None
    desc.seed = d.desc.seed
    return desc, arrs


@pytest.mark.parametrize("dtype,P,Q,no_aut", [(0, 700, 1024, False), (1, 1024, 1024, True)])
def test_noalloc_matches_handle_api_on_consecutive_calls(dtype, P, Q, no_aut):
    from paper_2510_19764_gb300 import abi, build, net
    build.build()
    rag = synth.random_ragged(21, P, Q, 0.1, no_autapse=no_aut)
    rng = np.random.default_rng(2)
    d = net.DeviceRagged(rag.row_len, rag.ind, rag.w, Q, dtype=dtype, no_autapse=no_aut, adam=True, deepr=True,
                         seed=31, m=rng.normal(size=rag.w.shape), v=rng.random(rag.w.shape))
    desc, arrs = _plain_copy(d)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for ridx in range(2):                      # two calls in a row share the static scratch
        drift = torch.as_tensor(rng.normal(0, 0.2, rag.w.shape), dtype=d.w.dtype, device="cuda")
        d.w += drift
        arrs["w"] += drift
        s_ref = torch.zeros(4, dtype=torch.int64, device="cuda")
        s_new = torch.zeros(4, dtype=torch.int64, device="cuda")
        abi.snn_rewire_deepr(d.handle, ridx, s_ref)
        abi.snn_rewire_deepr_noalloc(desc, ridx, s_new, status)
        torch.cuda.synchronize()
        assert torch.equal(s_ref, s_new)
        assert int(s_ref[0]) > 0
        assert torch.equal(d.row_len, arrs["row_len"])
        mask = (torch.arange(d.C, device="cuda")[None] < d.row_len[:, None])
        for k in ("ind", "w", "m", "v"):
            assert torch.equal(getattr(d, k)[mask], arrs[k][mask]), k
        assert torch.equal(d.conn_bits, arrs["conn_bits"])
    assert int(status.item()) == 0
    assert d.status() == abi.SNN_OK


def test_noalloc_rejects_too_many_rows():
    from paper_2510_19764_gb300 import abi, build
    build.build()
    desc = abi.RaggedDesc()
    desc.P, desc.Q, desc.C, desc.dtype = 16385, 8, 4, 0
    with pytest.raises(abi.SnnError) as e:
        abi.snn_rewire_deepr_noalloc(desc, 0)
    assert e.value.status == abi.SNN_EINVAL
    assert "16384" in abi.snn_last_error()
    # a descriptor the handle API refuses (reserved != 0) is refused here too
    desc.P, desc.reserved = 8, 1
    with pytest.raises(abi.SnnError) as e:
        abi.snn_rewire_deepr_noalloc(desc, 0)
    assert e.value.status == abi.SNN_EINVAL
    assert "reserved" in abi.snn_last_error()
