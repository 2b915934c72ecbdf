"""Host logic of the pinned-memory pipeline: its chunk boundaries tile [0, n) exactly,
in order, with the last chunk's worth split into the requested number of pieces (no GPU:
the boundaries are computed before any copy or lookup is queued)."""
import pytest

from paper_2305_05810_gb300.pipeline import HostPipeline


def chunks(n, chunk, tail):
    p = HostPipeline.__new__(HostPipeline)      # boundaries only: no device, no streams
    p.chunk, p.tail = chunk, tail
    return p._chunks(n)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 4095, 4096, 4097, 33177600])
@pytest.mark.parametrize("chunk", [1, 4, 4096, 1 << 22])
@pytest.mark.parametrize("tail", [1, 2, 4, 7])
def test_chunks_tile_the_batch(n, chunk, tail):
    if n // chunk > 100000:
        pytest.skip("more chunks than a real call would use")
    c = chunks(n, chunk, tail)
    if n == 0:
        assert c == []
        return
    assert c[0][0] == 0 and c[-1][1] == n
    assert all(a < b for a, b in c)
    assert all(c[i][1] == c[i + 1][0] for i in range(len(c) - 1))
    assert all(b - a <= chunk for a, b in c)
    regular = -(-n // chunk)
    if tail == 1 or regular == 1:
        assert len(c) == regular                   # a single chunk is never split
    else:
        last = n - (regular - 1) * chunk
        piece = -(-last // tail)                     # equal pieces, the final one shorter
        assert len(c) == regular - 1 + -(-last // piece)
        assert all(b - a == chunk for a, b in c[:regular - 1])
        assert all(b - a == piece for a, b in c[regular - 1:-1])


def test_dense_workload_chunks():
    """The benchmark's configuration: 33,177,600 queries in 4M chunks, the last split in four."""
    c = chunks(33177600, 1 << 22, 4)
    assert len(c) == 7 + 4
    assert max(b - a for a, b in c[7:]) == 954368
