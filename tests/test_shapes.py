"""Launch shapes on the host (hjlo_shape_query, no GPU): over a sweep of line
lengths, line counts, windows, storage types and both searches, every shape
keeps the limits and the index ranges the pass kernel relies on -- threads
and shared memory within a CTA's, lanes' segments covering the rows searched,
and for row blocks: blocks covering the line, a block's staged span (its rows
+ weff - 1) no longer than the line (one wrap at most when gathering), every
row of a block inside its line, and tiles covering every launched line."""
import itertools

import pytest

NS = [1, 2, 3, 33, 100, 700, 1024, 4096, 8192, 16384, 40000, 262144]
LINES = [1, 3, 40, 200, 1024]
WEFFS = [1, 3, 21, 65, 129, 291, 1637, None]          # None: the full torus window (weff = N)


@pytest.fixture(autouse=True)
def _no_overrides(monkeypatch):
    for k in ("HJLO_LANES_PER_LINE", "HJLO_LINES_PER_TILE", "HJLO_OFFLOAD", "HJLO_BLOCK_ROWS"):
        monkeypatch.delenv(k, raising=False)


def _cases():
    for N, lines, w in itertools.product(NS, LINES, WEFFS):
        weff = N if w is None else w
        if weff > N or N * lines > (1 << 26):
            continue
        yield N, lines, weff


@pytest.mark.parametrize("algo", [1, 2], ids=["brute", "monge"])
@pytest.mark.parametrize("esize", [8, 4])
@pytest.mark.parametrize("num_sms,smem", [(152, 232448), (20, 101376)])
def test_shape_invariants(algo, esize, num_sms, smem):
    from paper_1210_4090_gb300 import hjlo
    ok = refused = 0
    for N, lines, weff in _cases():
        try:
            s = hjlo.shape_query(N, lines, weff, esize, algo, num_sms, smem)
        except hjlo.HjloError as e:
            assert e.status == 6, e                       # only "does not fit" may refuse
            # refused only when a whole line does not fit and row blocks cannot help
            assert 4 * weff > N or N > 1000, (N, lines, weff)
            refused += 1
            continue
        ok += 1
        case = (N, lines, weff, s)
        assert 32 <= s["threads"] <= 1024 and s["threads"] % 32 == 0, case
        assert 0 < s["smem_bytes"] <= smem, case
        assert s["threads"] == s["lanes_per_line"] * s["lines_per_tile"], case
        blocks, R, L = s["row_blocks"], s["block_rows"], s["line_points"]
        assert blocks >= 1
        if blocks > 1:
            if algo == 2:
                assert 4 * weff <= N, case                    # only windows up to a quarter of the line
                assert R >= max(1, weff - 1), case
            else:
                # brute force: wider windows only on an axis with few lines
                assert 4 * weff <= N or 2 * lines < num_sms, case
                assert R >= 1, case
            assert (blocks - 1) * R < N <= blocks * R, case     # blocks cover the line, none empty
            assert L == R + weff - 1 <= N, case               # the span wraps at most once
            rows = R
        else:
            assert R == 0 and L == N, case
            rows = N
        assert weff <= L, case
        assert s["tiles"] * s["lines_per_tile"] >= lines * blocks, case
        assert (s["tiles"] - 1) * s["lines_per_tile"] < lines * blocks, case
        if algo == 2:
            S = s["segment_rows"]
            assert S % 2 == 1 and s["lanes_per_line"] * S >= rows, case
            assert s["lanes_per_line"] <= L, case           # staging: at most one point per lane per sweep
        else:
            assert s["segment_rows"] == 1, case
    assert ok > 100 and refused >= 1


@pytest.mark.parametrize("num_sms,smem", [(152, 232448), (20, 101376)])
def test_decomposition_shape_invariants(num_sms, smem):
    """The decomposition pass: one CTA per line or row block, shared memory
    within the CTA's, and for row blocks the blocks cover the line and a
    block's span of sources (its rows + weff - 1) is no longer than the line,
    as its gather (one wrap at most) needs; a line that fits neither runs
    across CTAs, its write-back blocks covering the line."""
    from paper_1210_4090_gb300 import hjlo
    ok = split = 0
    for N, lines, weff in _cases():
        try:
            s = hjlo.shape_query(N, lines, weff, 8, 3, num_sms, smem)
        except hjlo.HjloError as e:
            assert e.status == 6, e
            continue
        ok += 1
        case = (N, lines, weff, s)
        assert s["threads"] in (256, 1024) and 0 < s["smem_bytes"] <= smem, case
        blocks, R, L = s["row_blocks"], s["block_rows"], s["line_points"]
        if s["split_chunks"]:
            # a line that fits neither one CTA nor row blocks: its period cut
            # into chunks across CTAs, the outputs in blocks of split_rows
            split += 1
            V = s["split_rows"]
            assert blocks == 1 and R == 0 and 1 <= V <= N, case
            assert s["split_chunks"] * 4096 >= N + weff - 1 > (s["split_chunks"] - 1) * 64, case
            assert s["tiles"] == lines * -(-N // V), case
            continue
        assert s["split_rows"] == 0, case
        assert s["tiles"] == lines * blocks, case
        if blocks > 1:
            assert 4 * weff <= N and R >= max(1, weff - 1), case
            assert (blocks - 1) * R < N <= blocks * R, case
            assert L == R + weff - 1 <= N, case
        else:
            assert R == 0 and L == N, case
    assert ok > 50 and split >= 1


def test_shape_query_rejects_bad_arguments():
    from paper_1210_4090_gb300 import hjlo
    for args in [(0, 1, 1), (10, 0, 1), (10, 1, 0), (10, 1, 11)]:
        with pytest.raises(hjlo.HjloError) as e:
            hjlo.shape_query(*args)
        assert e.value.status == 1
    with pytest.raises(hjlo.HjloError):
        hjlo.shape_query(100, 1, 5, esize=2)
    with pytest.raises(hjlo.HjloError):
        hjlo.shape_query(100, 1, 5, algo=4)
    with pytest.raises(hjlo.HjloError):
        hjlo.shape_query(100, 1, 5, esize=4, algo=3)     # the decomposition pass runs in binary64
