"""Failure detection without a GPU fault: every device-side spin wait of the
reconstruction queue is bounded by the pipe's cycle budget.  With a budget of
a few hundred cycles the idle workers give up, the kernel returns, the
status word reports PIPE_ETIMEOUT, and the context stays usable: a pipe with
the normal budget then matches the oracle on the same tile."""
import numpy as np
import pytest

import synth
from tests.gpu_util import assert_planes_equal, oracle_all, run_gpu

pytestmark = pytest.mark.gpu


def test_wait_budget_exhaustion_is_reported_and_recoverable():
    import paper_1209_3332_gb300 as P
    from paper_1209_3332_gb300 import build
    build.build()
    rgb = synth.tile(1024, 1024, 61, n_nuclei=200, frac_cluster=0.2)
    tight = P.Pipe(0, wait_budget_cycles=300)
    run_gpu(tight, rgb, want_planes=False)
    assert tight.status() == P.PIPE_ETIMEOUT
    assert tight.status() == P.PIPE_OK  # reading the status clears it
    tight.close()
    normal = P.Pipe(0)
    g = run_gpu(normal, rgb)
    assert_planes_equal(g, oracle_all(rgb))
    assert normal.status() == P.PIPE_OK
    normal.close()
