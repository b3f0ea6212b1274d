"""CPU oracle of the EconoJax hot path (arxiv 2410.22165).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports it and shares no code
with it.

* :mod:`oracle.env` - the environment rules (Section 3), in plain C, one
  environment at a time, double-precision reporting track plus a float
  decision mirror.
"""
