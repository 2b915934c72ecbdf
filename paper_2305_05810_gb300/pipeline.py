"""Lookups on host-resident queries, pipelined across CUDA streams.

A batch whose coordinates (and levels of detail) live in pinned host memory and whose
results are wanted in pinned host memory is split into chunks; chunk c runs on
stream c mod S as host-to-device copy, one library lookup (query_offset advanced by the
chunk's start, so the variates and results are those of one call over the whole
batch) and device-to-host copy.  Copies of one chunk overlap the lookups and copies of
others (the copy engines run both directions concurrently).  Each stream reuses its
own device buffers, which the stream's ordering keeps safe.  The call is asynchronous
with respect to the host and ordered on the caller's current stream: the streams wait
for the work already queued there, and the current stream waits for them at the end.
"""
import paper_2305_05810_gb300 as stf


class HostPipeline:
    """tail: the last chunk's worth of queries is split into this many smaller chunks, so
    that the lookup and device-to-host copy left after the final host-to-device copy
    are short."""

    def __init__(self, texture, chunk=1 << 22, n_streams=3, device=None, tail=1):
        import torch
        self.torch = torch
        self.tex = texture
        self.chunk = int(chunk)
        self.tail = max(1, int(tail))
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_streams)]
        self.bufs = [{} for _ in range(n_streams)]

    def _buf(self, k, name, shape, dtype):
        b = self.bufs[k].get(name)
        n = 1
        for d in shape:
            n *= d
        if b is None or b.numel() < n:
            with self.torch.cuda.stream(self.streams[k]):
                b = self.torch.empty(n, dtype=dtype, device=self.device)
            self.bufs[k][name] = b
        return b[:n].view(*shape)

    def _chunks(self, n):
        """[a, b) ranges covering 0..n: chunks of self.chunk, the last chunk's worth split
        into self.tail pieces."""
        edges = list(range(0, n, self.chunk)) + [n]
        if self.tail > 1 and len(edges) > 2:
            a = edges[-2]
            step = -(-(n - a) // self.tail)
            edges = edges[:-2] + list(range(a, n, step)) + [n]
        return list(zip(edges[:-1], edges[1:]))

    def lookup(self, params, h_coords, h_out, h_lod=None, stochastic=True):
        """Filter every query of h_coords (n x 2 or n x 3, pinned) into h_out
        (n x channels, pinned) with the given stf_lookup_params."""
        torch = self.torch
        n = h_coords.shape[0]
        d = h_coords.shape[1]
        C = h_out.shape[1]
        cur = torch.cuda.current_stream(self.device)
        for s in self.streams:
            s.wait_stream(cur)
        for c, (a, b) in enumerate(self._chunks(n)):
            k = c % len(self.streams)
            s = self.streams[k]
            m = b - a
            with torch.cuda.stream(s):
                d_in = self._buf(k, "coords", (m, d), torch.float32)
                d_in.copy_(h_coords[a:b], non_blocking=True)
                d_lod = None
                if h_lod is not None:
                    d_lod = self._buf(k, "lod", (m,), torch.float32)
                    d_lod.copy_(h_lod[a:b], non_blocking=True)
                d_out = self._buf(k, "out", (m, C), torch.float32)
                p = stf.LookupParams.from_buffer_copy(params)
                p.query_offset = params.query_offset + a
                if stochastic:
                    stf.stf_lookup_batch(self.tex.handle, p, d_in, d_lod, m, d_out, None, s)
                else:
                    stf.stf_lookup_batch_deterministic(self.tex.handle, p, d_in, d_lod, m, d_out, s)
                h_out[a:b].copy_(d_out, non_blocking=True)
        for s in self.streams:
            cur.wait_stream(s)
        return h_out
