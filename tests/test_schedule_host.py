"""Host logic of the single-problem schedule of the tensor-core passes (no GPU).

The loader warp of CTA i walks, chunk by chunk of `chunk` streamed blocks, the pairs
[i W / g, (i + 1) W / g) of the chunk's flattened (row block, streamed block) space and writes
each run (a maximal piece of one row block) to partial slot slot_base[c][o] + i. The reduction
then sums the first nslot[o] slots of row block o. This walks that schedule by brute force and
checks the library's layout against it: every slot a row block's reduction reads is written by
exactly one run, and the runs of a row block cover its streamed blocks exactly once. It also
checks the automatic chunk width against the 32 MiB budget and the one-pair-per-CTA rule."""
import numpy as np
import pytest

from paper_2604_09233_gb300 import native


def _walk(n_outer, n_inner, chunk, g, base):
    written = {}
    for i in range(g):
        c = 0
        for c0 in range(0, n_inner, chunk):
            wc = min(chunk, n_inner - c0)
            w_total = n_outer * wc
            for w in range(i * w_total // g, (i + 1) * w_total // g):
                o, j = divmod(w, wc)
                slot = int(base[c, o]) + i
                written.setdefault((o, slot), []).append(c0 + j)
            c += 1
    return written


CASES = [
    (488, 3456, 576, 152),   # 3D E pass: 6 chunks
    (512, 280, 280, 152),    # 2D E^H pass: one chunk
    (280, 512, 512, 152),    # 2D E pass: one chunk
    (20, 37, 8, 16),         # ragged last chunk
    (3, 10, 4, 5),           # a CTA range inside one row block
    (12, 5, 2, 7),           # forced narrow chunks with a narrowed grid
    (1, 9, 1, 1),            # one row block, one CTA, width 1
]


@pytest.mark.parametrize("n_outer,n_inner,chunk,g", CASES)
def test_every_read_slot_is_written_once_and_covers_the_row_block(n_outer, n_inner, chunk, g):
    base, nslot, mx = native.sense_diag_stream_k_layout(n_outer, n_inner, chunk, g)
    assert mx == nslot.max() >= 1
    written = _walk(n_outer, n_inner, chunk, g, base)
    for o in range(n_outer):
        slots = sorted(s for (oo, s) in written if oo == o)
        assert slots == list(range(int(nslot[o]))), (o, slots, nslot[o])
        cover = sorted(j for s in slots for j in written[(o, s)])
        assert cover == list(range(n_inner)), o
        # a run is one contiguous piece of streamed blocks
        for s in slots:
            js = written[(o, s)]
            assert js == list(range(js[0], js[0] + len(js))), (o, s)


def test_a_chunk_without_a_pair_for_every_cta_is_rejected():
    with pytest.raises(native.SenseError):
        native.sense_diag_stream_k_layout(3, 10, 4, 7)   # last chunk: 3 x 2 pairs < 7 CTAs


@pytest.mark.parametrize("cp", [8, 16, 32, 64])
def test_automatic_chunk_width(cp):
    per_block = 2 * 2 * 2 * cp * 128 + 16384
    budget = 32 << 20
    # the 2D voxel side (512 blocks): one chunk while its images fit the budget
    w512 = native.sense_diag_chunk_width(280, 512, cp, 152)
    assert (w512 == 512) == (512 * per_block <= budget)
    # the 3D voxel side: chunks under the budget, equal but for the last, each with a pair per CTA
    for n_outer, n_inner in ((488, 3456), (100, 20000), (2, 5000)):
        w = native.sense_diag_chunk_width(n_outer, n_inner, cp, 152)
        nch = -(-n_inner // w)
        last = n_inner - (nch - 1) * w
        if n_inner * per_block <= budget:
            assert w == n_inner
        elif w < n_inner:
            # equal chunks of at most the budget (rounding adds at most one block)
            assert w * per_block <= budget + per_block and n_outer * last >= 152
        else:
            # the budget's chunking would leave a CTA without a pair: one chunk instead
            n0 = -(-n_inner * per_block // budget)
            w0 = -(-n_inner // n0)
            last0 = n_inner - (-(-n_inner // w0) - 1) * w0
            assert n_outer * last0 < 152
    with pytest.raises(native.SenseError):
        native.sense_diag_chunk_width(0, 10, cp, 152)
