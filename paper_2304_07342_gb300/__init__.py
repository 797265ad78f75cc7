"""GB300-native chunked multi-byte LZSS (gpuLZ method) -- package root.

The CUDA library is loaded lazily, on first use, by :mod:`.lz`; importing
the package itself needs no GPU (so the input generators in :mod:`.synth`
can be used anywhere).  There is no CPU fallback: every entry point in
:mod:`.lz` raises if the compiled library is missing.
"""
