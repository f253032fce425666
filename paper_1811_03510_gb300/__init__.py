"""GB300 (sm_103a) closest-hit ray intersection with Catmull-Clark subdivision surfaces given as bicubic
Bezier and Gregory patches (Binder & Keller, arXiv 1811.03510).  The compute path is libccs.so
(csrc/, C ABI in include/ccs.h); `ccs` is its Python binding and `scenegen` the synthetic inputs."""
