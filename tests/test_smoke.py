"""The entry point's smoke() on cuda:0: one small call of the denoiser
(Algorithms 1-2 iterated, Section 2) that must match the oracle in every
pixel, k and the converged flag."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_matches_oracle(capsys):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_5390_gb300 import build
    build.build()
    import __graft_entry__
    __graft_entry__.smoke()
    assert "bit-exact vs oracle" in capsys.readouterr().out
