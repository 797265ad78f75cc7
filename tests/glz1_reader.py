"""Independent pure-Python reader of the GLZ1 stream layout.

Written from the layout description (header, chunk table, superblock index,
per-chunk records of flags then payload) for the tests only.  It shares no
code with the C oracle or the CUDA library, so a test can decode either
side's bytes into tokens and check them against brute force.
"""
from __future__ import annotations

import struct
from dataclasses import dataclass, field


@dataclass
class Stream:
    S: int
    offB: int
    m: int
    M: int
    C: int
    W: int
    n_chunks: int
    n_bytes: int
    table: list = field(default_factory=list)      # (n_tokens, payload_bytes)
    index: list = field(default_factory=list)      # u64 per 64 chunks
    records_at: int = 0
    record_offsets: list = field(default_factory=list)  # relative to records_at
    tokens: list = field(default_factory=list)     # per chunk [(len, off)]
    stored: list = field(default_factory=list)     # per chunk: stored as is (version 2)
    total_bytes: int = 0
    version: int = 1
    overlap: bool = False


def read(buf: bytes) -> Stream:
    buf = bytes(buf)
    assert buf[:4] == b"GLZ1", "magic"
    ver, S, offB, m, M = buf[4], buf[5], buf[6], buf[7], buf[8]
    assert ver in (1, 2) and buf[9] <= (1 if ver == 2 else 0) and buf[10:12] == b"\0\0"
    C, W, nc = struct.unpack_from("<III", buf, 12)
    (n,) = struct.unpack_from("<Q", buf, 24)
    st = Stream(S, offB, m, M, C, W, nc, n)
    st.version = ver
    st.overlap = buf[9] == 1
    pos = 32
    for c in range(nc):
        st.table.append(struct.unpack_from("<II", buf, pos))
        pos += 8
    for j in range((nc + 63) // 64):
        st.index.append(struct.unpack_from("<Q", buf, pos)[0])
        pos += 8
    st.records_at = pos
    rel = 0
    for c in range(nc):
        ntok, pay = st.table[c]
        st.record_offsets.append(rel)
        if ver == 2 and ntok == 0:  # stored chunk: its bytes, no flags
            bytes_c = min(C, n - c * C)
            assert pay == bytes_c, "stored chunk size"
            assert len(buf[pos + rel: pos + rel + pay]) == pay, "truncated record"
            st.tokens.append([])
            st.stored.append(True)
            rel += pay
            continue
        st.stored.append(False)
        fb = (ntok + 7) // 8
        rec = buf[pos + rel: pos + rel + fb + pay]
        assert len(rec) == fb + pay, "truncated record"
        flags, payload = rec[:fb], rec[fb:]
        toks = []
        q = 0
        for t in range(ntok):
            if (flags[t // 8] >> (t % 8)) & 1:
                ln = payload[q]
                off = payload[q + 1] if offB == 1 else payload[q + 1] | (payload[q + 2] << 8)
                toks.append((ln, off + 1))
                q += 1 + offB
            else:
                toks.append((1, 0))
                q += S
        tail = min(C, n - c * C) % S if ver == 2 else 0  # version 2: bytes after the last symbol
        assert q + tail == pay, "payload size mismatch"
        # padding bits of the last flag byte are zero
        if ntok % 8:
            assert flags[-1] >> (ntok % 8) == 0, "nonzero pad bits"
        st.tokens.append(toks)
        rel += fb + pay
    st.total_bytes = pos + rel
    return st


def literal_bytes(buf: bytes, st: Stream, c: int):
    """Payload bytes of each literal of chunk c, in token order."""
    buf = bytes(buf)
    ntok, pay = st.table[c]
    base = st.records_at + st.record_offsets[c] + (ntok + 7) // 8
    q = 0
    out = []
    for ln, off in st.tokens[c]:
        if off:
            q += 1 + st.offB
        else:
            out.append(buf[base + q: base + q + st.S])
            q += st.S
    return out
