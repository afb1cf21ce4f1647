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
