"""The chunk pipeline of the double-word moment kernel, replayed on the host.

The kernel (k_moments_dw) runs, in one interval between two CTA barriers, the row constants
of chunk t+1, alpha of chunk t, phase B of chunk t-1, phase C of chunk t-2 and phase D of the
plane whose last chunk was t-3, on buffers indexed by chunk parity (row constants, alpha,
T1) and plane parity (T2).  This test walks the same schedule for every G the library
accepts and checks that no buffer is written and read by different steps in one interval,
that every read sees the data of the chunk (or plane) it needs, and that the moments end
complete.  The chunking is the kernel's: nb = max(1, min(G, 256 // (2 ceil(G/2)))) rows of
one plane, a lane pair per mirrored pair of points of a row."""
import pytest


def schedule_ok(G, chunk=256):
    lanes_per_row = 2 * ((G + 1) // 2)
    nb = max(1, min(G, chunk // lanes_per_row))
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
