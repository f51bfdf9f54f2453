"""Concurrent use of the library: independent plans driven from separate host threads on separate
streams (the way bench.py and the request server run several passes at once) give exactly the
results of one plan run alone."""
import threading

import numpy as np
import pytest

import synth
from tests.gpu_util import to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def test_concurrent_plans_match_a_single_plan(bnd):
    torch = torch_cuda()
    p = synth.delay_2d(s=24, seed=2)
    split = bnd.Split.from_problem(p)
    Vs = [synth.random_probe_block(p.n, p.L, k) for k in range(3)]
    Vd = [to_dev(np.asfortranarray(V), torch) for V in Vs]
    # reference: one plan, one stream, the three probe blocks in turn
    ref = []
    plan = bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1)
    for V in Vd:
        plan.execute(V)
        torch.cuda.synchronize()
        ref.append(plan.result())
    # three plans on three streams from three threads, two passes each
    plans = [bnd.Plan(split, p.region, p.N, p.L, p.M, precision=1) for _ in range(3)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    errors = []

    def run(i):
        try:
            for _ in range(2):
                plans[i].execute(Vd[i], streams[i].cuda_stream)
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    assert not errors, errors
    for i in range(3):
        got = plans[i].result()
        assert len(got["lam"]) == len(ref[i]["lam"]) > 0
        assert np.array_equal(got["lam"], ref[i]["lam"])
        assert np.array_equal(got["X"], ref[i]["X"])
        assert np.array_equal(got["eta"], ref[i]["eta"])
