"""GB300 pixel-track reconstruction: hit sort, doublets, cellular-automaton connection, ntuplets
and broken-line (or Riemann) fits, batched over many events, with optional track selection,
track covariances and primary vertices.

Modules:
  pxr        the binding of the C ABI in include/pxr.h (contexts, serving, device-resident plans,
             the fit-only and allocation-free entry points); all computation runs in libpxr.so
  build_lib  builds libpxr.so in-tree with nvcc for sm_103a
  autotune   picks the phi-bin count and per-stage grid sizes on a caller's batch
  shard      event sharding over ranks (no collective)
  synth      seeded synthetic events, batches, ntuplets and serving streams
"""
