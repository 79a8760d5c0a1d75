"""The pipelined host-buffer entry point (epic_image_host_async + epic_host_wait):
several integrations queued back to back through the two upload / download
slots give, each, the image the synchronous host-buffer call gives (bitwise: the
same plan and graph), and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err

pytestmark = pytest.mark.gpu


def _inputs(wl, seed):
    rng = np.random.default_rng(seed)
    v = synth.random_ci4(wl.v.shape, rng)
    return torch.from_numpy(v).pin_memory()


@pytest.mark.parametrize("precision", [epic.EPIC_FP32, epic.EPIC_TC_SPLIT_FP16])
def test_queued_integrations_match_the_synchronous_call(precision):
    wl = synth.random_small(A=64, P=2, C=3, T=9, N=128, K=5, seed=901)
    plan = epic.Plan.from_workload(wl, precision=precision)
    g = torch.from_numpy(wl.gains).pin_memory()
    vs = [_inputs(wl, 910 + i) for i in range(5)]
    outs = [torch.empty(plan.out_floats // 2, dtype=torch.complex64).pin_memory() for _ in range(5)]
    for v, o in zip(vs, outs):          # five calls queued before any wait: both slots reused
        plan.image_host_async(v, g, out=o)
    plan.host_wait()
    for i, (v, o) in enumerate(zip(vs, outs)):
        ref = plan.image_host(v, g)
        assert torch.equal(o, ref), i
    # one of them against the oracle
    wl.v = vs[3].numpy()
    err = peak_rel_err(outs[3].numpy(), oracle.workload_image(wl), wl.grid_n, 2)
    assert err.max() < 1e-5
    assert plan.status() == epic.EPIC_OK
    plan.close()


def test_queued_calls_with_and_without_gains_and_empty():
    wl = synth.random_small(A=40, P=2, C=2, T=6, N=64, K=3, seed=920)
    plan = epic.Plan.from_workload(wl)
    v = torch.from_numpy(wl.v).pin_memory()
    g = torch.from_numpy(wl.gains).pin_memory()
    a = plan.image_host_async(v, g)
    b = plan.image_host_async(v, None)
    c = plan.image_host_async(v[:0].contiguous(), g)
    plan.host_wait()
    assert torch.equal(a, plan.image_host(v, g))
    assert torch.equal(b, plan.image_host(v, None))
    assert torch.count_nonzero(c) == 0
    plan.close()


def test_async_rejects_bad_arguments():
    wl = synth.random_small(A=16, P=2, C=1, T=4, N=64, K=3, seed=930)
    plan = epic.Plan.from_workload(wl)
    v = torch.from_numpy(wl.v)
    with pytest.raises(ValueError):
        plan.image_host_async(v.cuda())          # device input to the host entry point
    too_many = torch.zeros((wl.T + 1, wl.C, wl.A, wl.n_pol), dtype=torch.uint8)
    with pytest.raises(epic.EpicError):
        plan.image_host_async(too_many)
    plan.host_wait()
    plan.close()
