"""Host-in, host-out batched calls with the copies overlapped with the computation.

A batch held in pinned host memory is split into chunks along its leading (batch) dimension; chunk
c is copied to the device on one stream, computed on a second and copied back on a third, so that
the transfer of chunk c + 1 and the read-back of chunk c - 1 run while chunk c is computed.  The
library calls themselves are the ordinary batched entry points on device views of each chunk;
this module only orders streams and events (the paper processes batches already on the GPU, so it
has no counterpart)."""
from __future__ import annotations


def chunk_bounds(n: int, chunks: int):
    """[(c0, c1), ...]: at most ``chunks`` consecutive, non-empty ranges covering 0 .. n - 1, all of
    the same length but the last."""
    if n <= 0:
        return []
    chunks = max(1, min(chunks, n))
    step = (n + chunks - 1) // chunks
    return [(c0, min(c0 + step, n)) for c0 in range(0, n, step)]


class ChunkPipeline:
    """Device buffers and streams for repeated host -> device -> host runs of one batch shape.

    ``h_in`` / ``h_out``: pinned host tensors whose leading dimension is the batch; ``d_in`` /
    ``d_out``: device tensors of the same shapes (owned by the caller, reused on every run).
    ``compute(c0, c1, d_in_views, d_out_views, stream)`` enqueues the library calls for batch
    entries c0 .. c1 - 1 on ``stream``."""

    def __init__(self, h_in, h_out, d_in, d_out, compute, chunks: int = 4):
        import torch
        self.h_in, self.h_out, self.d_in, self.d_out = list(h_in), list(h_out), list(d_in), list(d_out)
        for h in self.h_in + self.h_out:
            if not h.is_pinned():
                raise ValueError("host buffers must be pinned")
        self.compute = compute
        self.bounds = chunk_bounds(self.h_in[0].shape[0], chunks)
        dev = self.d_in[0].device
        self.s_in, self.s_comp, self.s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
        self.ev_in = [torch.cuda.Event() for _ in self.bounds]
        self.ev_comp = [torch.cuda.Event() for _ in self.bounds]

    def run(self, stream=None):
        """One host -> device -> host pass over the whole batch; ordered after ``stream`` (default:
        the current stream), which in turn waits for the last read-back."""
        import torch
        caller = stream or torch.cuda.current_stream()
        for s in (self.s_in, self.s_comp, self.s_out):
            s.wait_stream(caller)
        for c, (c0, c1) in enumerate(self.bounds):
            with torch.cuda.stream(self.s_in):
                for d, h in zip(self.d_in, self.h_in):
                    d[c0:c1].copy_(h[c0:c1], non_blocking=True)
                self.ev_in[c].record(self.s_in)
            self.s_comp.wait_event(self.ev_in[c])
            self.compute(c0, c1, [d[c0:c1] for d in self.d_in], [d[c0:c1] for d in self.d_out], self.s_comp)
            self.ev_comp[c].record(self.s_comp)
            self.s_out.wait_event(self.ev_comp[c])
            with torch.cuda.stream(self.s_out):
                for h, d in zip(self.h_out, self.d_out):
                    h[c0:c1].copy_(d[c0:c1], non_blocking=True)
        caller.wait_stream(self.s_out)
        caller.wait_stream(self.s_comp)
