"""The request loop on the GPU: every served request's final state equals the same request
run alone for the same number of steps (bitwise), with requests arriving while others run."""
import numpy as np
import pytest

from paper_1810_08137_gb300 import inputs as I
from paper_1810_08137_gb300 import serve

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone_runs():
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    cfgs = [I.channel_config(nx=12, ny=6, n_vel=12, kn=0.2, rho_in=1.1, name="s0"),
            I.channel_config(nx=20, ny=10, n_vel=16, kn=0.02, rho_in=1.3, name="s1"),
            I.channel_config(nx=9, ny=5, n_vel=21, kn=1.0, rho_in=1.05, name="s2"),
            I.channel_config(nx=14, ny=7, n_vel=10, kn=0.005, rho_in=1.4, name="s3")]
    prims = [I.initial_prim(c, I.seed_for(5, k)) for k, c in enumerate(cfgs)]
    reqs = serve.make_requests(cfgs, [0.0, 0.0, 0.02, 0.05], prims)
    need = max(ugks.state_bytes(c, ugks.FP32F) for c in cfgs)
    srv = serve.gpu_server(hbm_budget=3 * need, max_slots=3, tol=1e-4, max_steps=400,
                           check_every=10, keep_state=True)
    st = srv.run(reqs)
    srv.batch_handle.close()
    s = st.summary()
    assert s["finished"] == 4
    for r in reqs:
        with ugks.Solver(r.cfg, ugks.FP32F) as a:
            a.init_maxwellian(*r.prim)
            a.step(r.steps)
            f, W = a.get_state()
        assert np.array_equal(f, r.state[0]) and np.array_equal(W, r.state[1]), r.cfg.name
