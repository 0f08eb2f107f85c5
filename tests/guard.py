"""Guard bands around device outputs (the sanitizer substitute for tests).

`guarded(shape, dtype, fill)` returns a CUDA tensor of `shape` that sits in the
middle of a larger byte buffer; the GUARD bytes on either side hold the
sentinel byte 0xA5.  After a call, `check()` asserts that every guard byte is
unchanged, so a store past either end of the output (a ragged tail written one
vector too far, a row index off by one, a partial written to the wrong slot)
fails the test instead of silently corrupting a neighbour.  The guard is 4 KiB
on each side: larger than any vector store, and a multiple of 256 bytes so the
output keeps the base allocation's alignment.
"""
import math

import numpy as np
import torch

GUARD = 4096
SENTINEL = 0xA5


class Guarded:
    def __init__(self, shape, dtype, fill=0, device="cuda"):
        shape = tuple(int(s) for s in (shape if isinstance(shape, (tuple, list)) else (shape,)))
        isz = torch.empty(0, dtype=dtype).element_size()
        self.nbytes = math.prod(shape) * isz
        self.buf = torch.full((GUARD + self.nbytes + GUARD,), SENTINEL, dtype=torch.uint8, device=device)
        inner = self.buf[GUARD:GUARD + self.nbytes]
        self.t = inner.view(dtype).view(shape) if self.nbytes else torch.empty(shape, dtype=dtype, device=device)
        if self.nbytes:
            self.t.fill_(fill)

    def check(self, what=""):
        b = self.buf.cpu().numpy()
        head, tail = b[:GUARD], b[GUARD + self.nbytes:]
        bad_h = np.flatnonzero(head != SENTINEL)
        bad_t = np.flatnonzero(tail != SENTINEL)
        assert bad_h.size == 0, "%s: %d guard bytes before the output overwritten (nearest at -%d)" % (
            what, bad_h.size, GUARD - bad_h.max())
        assert bad_t.size == 0, "%s: %d guard bytes after the output overwritten (first at +%d)" % (
            what, bad_t.size, bad_t.min())
        return self.t


def guarded(shape, dtype, fill=0):
    """A Guarded output: `.t` is the tensor to pass, `.check()` verifies the bands."""
    return Guarded(shape, dtype, fill)
