"""Host-side logic of the Python binding (no GPU): stream arguments reach chase_create as
the C ABI expects them."""
import paper_2603_10514_gb300 as P


class FakeLib:
    def __init__(self):
        self.streams = []

    def chase_create(self, hp, device, stream):
        self.streams.append(None if stream is None else stream.value)
        return 0

    def chase_destroy(self, h):
        return 0


def test_default_stream_is_passed_as_cuda_stream_legacy(monkeypatch):
    """torch's default stream has handle 0, which the C ABI reads as "make a stream of your
    own" (not ordered with the caller's work on the default stream); the binding passes
    cudaStreamLegacy for it instead."""
    fake = FakeLib()
    monkeypatch.setattr(P, "lib", lambda: fake)
    P.Handle(0, stream=0).close()
    P.Handle(0, stream=0x7F00AB).close()
    P.Handle(0).close()
    assert fake.streams == [P.CUDA_STREAM_LEGACY, 0x7F00AB, None]
    assert P.CUDA_STREAM_LEGACY == 1


def test_missing_library_raises_with_no_fallback(monkeypatch, tmp_path):
    """Without the built CUDA library every call fails loudly: there is no CPU path."""
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "libchase_gb300.so"))
    import pytest
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        P.lib()
    with pytest.raises(RuntimeError):
        P.Handle(0)


def test_product_sources_never_reach_the_oracle():
    """The package, its CUDA sources and the public header neither import, link nor load the
    oracle (test infrastructure only)."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pat = re.compile(r"\bimport oracle\b|\bfrom oracle\b|liboracle|chase_oracle|orc_[a-z]")
    hits = []
    for d in ("paper_2603_10514_gb300", "include"):
        for dirpath, dirnames, files in os.walk(os.path.join(root, d)):
            dirnames[:] = [x for x in dirnames if x not in ("_build", "__pycache__")]
            for f in files:
                if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                    text = open(os.path.join(dirpath, f), errors="replace").read()
                    if pat.search(text):
                        hits.append(os.path.join(d, f))
    assert hits == []
