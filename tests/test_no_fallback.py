"""The product path has no CPU fallback: without the built library the binding raises, and without
a usable GPU creating a context fails with the library's CUDA error instead of computing anything
on the host (no GPU needed for these checks)."""
import pytest

from paper_2503_22875_gb300 import ozg


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(ozg, "_lib", None)
    monkeypatch.setattr(ozg._build, "LIB", str(tmp_path / "libozg.so"))
    with pytest.raises(ImportError, match="not built"):
        ozg.load()


def test_context_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2503_22875_gb300 import build
    build.build()
    ozg.load()
    with pytest.raises(ozg.OzgError, match="CUDA"):
        ozg.Context()
