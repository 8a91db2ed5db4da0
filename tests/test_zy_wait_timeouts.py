"""Collected last: after every GPU test of the session (single-beam, batched,
pipelined and allocation-free executes), no kernel gave up a bounded wait on a
bulk copy (tx_wait_timeouts counts them on the device)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_no_kernel_gave_up_a_wait():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_13834_gb300 import build
    build.build()
    import paper_2401_13834_gb300 as tx
    assert tx.wait_timeouts() == 0
