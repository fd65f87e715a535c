"""The chunk pipeline of the double-word moment kernel, replayed on the host.

The kernel (k_moments_dw) runs, in one interval between two CTA barriers, the row constants
of chunk t+1, alpha of chunk t, phase B of chunk t-1, phase C of chunk t-2 and phase D of the
plane whose last chunk was t-3, on buffers indexed by chunk parity (row constants, alpha,
T1) and plane parity (T2).  This test walks the same schedule for every G the library
accepts and checks that no buffer is written and read by different steps in one interval,
that every read sees the data of the chunk (or plane) it needs, and that the moments end
complete.  The chunking is the kernel's, a lane pair per mirrored pair of points of a row:
at most cap = max(1, min(G, 256 // (2 ceil(G/2)))) rows of one plane per chunk, as few chunks
as that allows, the rows spread evenly over them: nb = ceil(G / ceil(G / cap))."""
import pytest

def rows_cap(G, chunk=256):
    return max(1, min(G, chunk // (2 * ((G + 1) // 2))))


def rows_per_chunk(G, chunk=256):
    cap = rows_cap(G, chunk)
    return -(-G // -(-G // cap))


def schedule_ok(G, chunk=256):
    nb = rows_per_chunk(G, chunk)
    ncp = (G + nb - 1) // nb
    T = G * ncp
    state = {}
    for step in range(-1, T + 3):
        reads, writes = [], []
        if step + 1 < T:
            writes.append((("row", (step + 1) & 1), ("rc", step + 1)))
        if 0 <= step < T:
            reads.append((("row", step & 1), ("rc", step)))
            writes.append((("alpha", step & 1), ("a", step)))
        tb, tc, td = step - 1, step - 2, step - 3
        if 0 <= tb < T:
            reads.append((("alpha", tb & 1), ("a", tb)))
            writes.append((("T1", tb & 1), ("b", tb)))
        if 0 <= tc < T:
            c, b0 = tc // ncp, (tc % ncp) * nb
            reads.append((("T1", tc & 1), ("b", tc)))
            if b0 > 0:
                reads.append((("T2", c & 1), ("c", tc - 1)))  # accumulation within a plane
            writes.append((("T2", c & 1), ("c", tc)))
        if 0 <= td < T and td % ncp == ncp - 1:
            p = td // ncp
            reads.append((("T2", p & 1), ("c", td)))
            if p > 0:
                reads.append((("I",), ("d", p - 1)))
            writes.append((("I",), ("d", p)))
        wbufs = [w[0] for w in writes]
        assert len(set(wbufs)) == len(wbufs)
        for buf, want in reads:
            read_modify_write = buf[0] == "I" or (buf[0] == "T2" and want == ("c", tc - 1))
            if not read_modify_write:
                assert buf not in wbufs, (G, step, buf)
            assert state.get(buf) == want, (G, step, buf, state.get(buf), want)
        for buf, what in writes:
            state[buf] = what
    return state[("I",)] == ("d", G - 1)


@pytest.mark.parametrize("G", range(1, 65))
def test_moment_pipeline_schedule(G):
    assert schedule_ok(G)


@pytest.mark.parametrize("G", range(1, 65))
def test_chunks_are_few_even_and_fit(G):
    # The chunking keeps the fewest chunks per plane that the 256 lanes allow, fits them,
    # and leaves no chunk emptier than it must: G = 24 gets 8 rows (three full chunks rather
    # than 10 + 10 + 4), G = 48 keeps 5 (ten chunks, the last of 3 rows).
    cap, nb = rows_cap(G), rows_per_chunk(G)
    ncp = -(-G // nb)
    assert ncp == -(-G // cap) and nb <= cap and nb * 2 * ((G + 1) // 2) <= max(256, 2 * ((G + 1) // 2))
    assert G - (ncp - 1) * nb >= G - (ncp - 1) * cap
    assert nb - (G - (ncp - 1) * nb) < ncp  # the last chunk is short by fewer rows than there are chunks
    if G in (24, 48):
        assert nb == {24: 8, 48: 5}[G]
