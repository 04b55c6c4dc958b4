"""The learned few-angle -> many-angle network, trained from scratch on the GPU at a
small size, beats the method without it (the few-angle volume scaled by the
least-squares gain) on scenes built from blocks it never saw."""
import pytest

pytestmark = pytest.mark.gpu


def test_training_gains_over_the_few_angle_volume():
    from paper_2604_06257_gb300 import build, learned
    build.build()
    net, rep = learned.train(n=32, bank_size=96, samples=384, epochs=4, batch=8, lr=1e-3, seed=1,
                             test_blocks=64, test_scenes=32, log=lambda *a: None)
    net.close()
    print(rep["untrained"], rep["trained"], rep["gain"])
    assert rep["untrained"]["network_db"] == pytest.approx(rep["untrained"]["few_angle_db"], abs=1e-3)
    assert rep["trained"]["network_db"] < rep["trained"]["few_angle_db"] - 1.0
