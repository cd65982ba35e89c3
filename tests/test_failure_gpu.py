"""Failure detection without a GPU fault: every bounded device wait gives up
after a limit and reports PHYLO_ETIMEOUT through the flag word.  A test-only
launch waits on an mbarrier nothing is armed on, with a limit of a few
rounds; the call returns the timeout status and the CUDA context stays
usable (an evaluation afterwards is still right)."""
import pytest

import synth
from parity import compare, oracle_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04390_gb300 import build as B
    B.build()


def test_bounded_wait_times_out_and_reports():
    from paper_2303_04390_gb300 import _native as N
    lib = N.load()
    s = torch.cuda.Stream()
    for rounds in (1, 4, 16):
        assert lib.phylo_selftest_bounded_wait(rounds, s.cuda_stream) == N.PHYLO_ETIMEOUT
    assert b"bounded wait" in lib.phylo_last_error(None)
    assert lib.phylo_selftest_bounded_wait(0, None) == N.PHYLO_EINVAL
    # the context is intact: an evaluation after the timeouts is right
    import paper_2303_04390_gb300 as pg
    w = synth.small_workload(12, 4, 4, 70, seed=36)
    ctx = pg.from_workload(w, "fp32")
    logL, grad = ctx.evaluate()
    ctx.close()
    compare(logL, grad, oracle_eval(w), "fp32", "after timeouts")
