"""A live context refuses bad arguments on the host, before any launch, and stays usable:
every entry point given NULL buffers (or called out of order) returns an error with a message,
and the next iteration is bit-identical to one run before the bad calls."""
import numpy as np
import pytest

from paper_1707_02342_gb300 import inputs
from tests import gpu_common as G
from tests import problems

pytestmark = pytest.mark.gpu


def test_bad_calls_leave_the_context_usable():
    from paper_1707_02342_gb300 import itmpc

    params, tmap, layers = G.small_workload(K=256, T=40)
    ctl = G.controller(params, tmap, layers)
    x0 = problems.x0_for(tmap, speed=2.5)
    U = inputs.nominal_controls(40, seed=8)
    before = G.run(ctl, x0, U, 2)
    assert before[3] == 0
    L, h = ctl._L, ctl._h
    calls = {
        "set_config": lambda: L.itmpc_set_config(h, None),
        "set_dynamics": lambda: L.itmpc_set_dynamics(h, 3, None, None, None, 1),
        "set_costmap": lambda: L.itmpc_set_costmap(h, None, 64, 64, 0.1, 0.0, 0.0, 1),
        "set_costmaps": lambda: L.itmpc_set_costmaps(h, 1, None, 64, 64, 0.1, 0.0, 0.0, 1),
        "iterate": lambda: L.itmpc_iterate(h, None, None, 0, None, None, None),
        "iterate_host": lambda: L.itmpc_iterate_host(h, None, None, 0, None, None, None),
        "noise": lambda: L.itmpc_noise(h, 0, None),
        "rollout_states": lambda: L.itmpc_rollout_states(h, None, None, 0, 1, None, None),
        "get_stats": lambda: L.itmpc_get_stats(h, None),
        "iterate_batch (not reserved)": lambda: L.itmpc_iterate_batch(h, 1, None),
        "batch_graph_launch (no graph)": lambda: L.itmpc_batch_graph_launch(h),
        "control_graph_launch (no graph)": lambda: L.itmpc_control_graph_launch(h),
        "control_step": lambda: L.itmpc_control_step(h, None, None, 0, 1, 1, None),
        "iterate_cem": lambda: L.itmpc_iterate_cem(h, None, None, 0, 0.8, None, None, None),
        "set_basis (network context)": lambda: L.itmpc_set_basis(h, None, 1),
        "update_from_noise": lambda: L.itmpc_update_from_noise(h, None, None, None, None),
        "iterate_fwd": lambda: L.itmpc_iterate_fwd(h, None, None, 0, 10, None, None, None, None, None),
        "iterate_bwd": lambda: L.itmpc_iterate_bwd(h, None, 0, 10, None, None, None, None, None, None, None, None,
                                                   None),
    }
    for name, call in calls.items():
        st = call()
        assert st in (itmpc.ERR_ARG, itmpc.ERR_STATE), (name, st)
        assert L.itmpc_last_error(h), name
    assert ctl.read_status() == 0
    after = G.run(ctl, x0, U, 2)
    assert after[3] == 0
    for a, b in zip(before[:3], after[:3]):
        np.testing.assert_array_equal(a, b)
    ctl.close()
