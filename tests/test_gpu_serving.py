"""GPU serving: requests run concurrently (continuous batching on separate
streams) give the same results as each request run alone."""
import numpy as np
import pytest

from paper_1502_03234_gb300 import slabgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,skin", [(0, None), (1, None), (1, 0.5)])
def test_results_same_alone_and_in_the_mix(prec, skin):
    import __graft_entry__

    __graft_entry__.build()
    from paper_1502_03234_gb300 import serving as sv

    spec = [(2048, 60), (9001, 40), (16000, 30), (4096, 80), (5001, 50)]
    slabs = [slabgen.make_slab(n, seed=100 + k, min_edge=17.0) for k, (n, _) in enumerate(spec)]

    def jobs():
        return [sv.Job(rid=k, n=n, nsteps=st, box=s.box, x=s.x, v=s.v, arrival=0.0)
                for k, ((n, st), s) in enumerate(zip(spec, slabs))]

    backend = sv.DcmBackend(precision=prec, skin=skin)
    mix = jobs()
    rep = sv.Server(backend, budget_bytes=8 << 30, max_slots=4, chunk_steps=10).run(mix, realtime=False)
    assert all(j.status == sv.DONE for j in mix), [j.error for j in mix]
    assert rep.max_active >= 2                           # work overlapped
    for k in range(len(spec)):
        alone = jobs()[k:k + 1]
        sv.Server(backend, budget_bytes=8 << 30, max_slots=1, chunk_steps=10).run(alone, realtime=False)
        xa, va, fa = alone[0].result
        xm, vm, fm = mix[k].result
        assert np.array_equal(xa, xm) and np.array_equal(va, vm) and np.array_equal(fa, fm)
    s = rep.summary()
    assert s["latency_s"]["p50"] > 0 and s["atom_steps_per_s"] > 0
