"""GB300-native VaPr path: batched FK -> sphere/cuboid collision cost with
self-collision -> joint gradients, with the large intermediate tensors stored
in ExMy formats (arXiv 2310.07854, Sec. III-IV).

The compute path is the CUDA library ``libvapr.so`` built from ``csrc/``;
``_lib`` is its thin ctypes binding.  ``synth`` draws seeded inputs and
``formats`` holds the host-side format logic.
"""
__all__ = ["synth", "formats"]
