"""The host path's chunk schedule (api._chunks): contiguous, covering, bounded, ramped."""
import pytest

from paper_2606_17065_gb300 import api


@pytest.mark.parametrize("n", [1, 255, 4096, 3 * 4096 + 77, 1 << 20, (1 << 21) + 5, 16777216, 5 * (1 << 21) - 3])
@pytest.mark.parametrize("ramp", [False, True])
def test_chunks_cover_rows_in_order(monkeypatch, n, ramp):
    monkeypatch.setattr(api, "HOST_RAMP", ramp)
    chunks = api._chunks(n)
    lo = 0
    for start, m in chunks:
        assert start == lo and 0 < m <= api.HOST_CHUNK
        lo += m
    assert lo == n


def test_ramp_halves_the_first_and_last_chunk(monkeypatch):
    monkeypatch.setattr(api, "HOST_RAMP", True)
    C = api.HOST_CHUNK
    sizes = [m for _, m in api._chunks(8 * C)]
    assert sizes[:4] == [C // 8, C // 8, C // 4, C // 2]
    assert sizes[-4:] == [C // 2, C // 4, C // 8, C // 8]
    assert sizes[4:-4] == [C] * 6
    monkeypatch.setattr(api, "HOST_RAMP", False)
    assert [m for _, m in api._chunks(8 * C)] == [C] * 8


def test_host_chunk_size_by_call_size():
    """Calls up to HOST_CHUNK / 4 rows take one unpipelined round trip; above, a quarter of the
    call per chunk (at least HOST_CHUNK / 8), and HOST_CHUNK from 4 HOST_CHUNK rows on."""
    C = api.HOST_CHUNK
    assert api._host_chunk(1) == 0 and api._host_chunk(C // 4) == 0
    assert api._host_chunk(C // 4 + 1) == C // 8
    assert api._host_chunk(C) == C // 4
    assert api._host_chunk(2 * C + 3) == -(-(2 * C + 3) // 4)
    assert api._host_chunk(4 * C) == C and api._host_chunk(16 * C) == C
    for n in (C // 4 + 1, C, 3 * C + 7):
        sizes = [m for _, m in api._chunks(n, api._host_chunk(n))]
        assert sum(sizes) == n and max(sizes) <= api._host_chunk(n)
