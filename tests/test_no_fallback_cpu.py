"""Without the CUDA library the package fails loudly: there is no CPU path to fall back
to (no GPU needed)."""
import pytest


def test_missing_library_raises(monkeypatch):
    from paper_2606_00444_gb300 import _abi, _build
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_build, "build", lambda *a, **k: "/nonexistent/libmeshgs.so")
    with pytest.raises(RuntimeError, match="missing"):
        _abi.lib()
    from paper_2606_00444_gb300 import MeshBVH
    with pytest.raises(RuntimeError, match="missing"):
        MeshBVH(10, 16, "cpu")
