"""FP64 CPU oracle of the clustered parametric spectral likelihood, its gradient, the fit and the
W.d reconstruction (arxiv 2604.08463, Sec. 2.1-2.4 and Sec. 3.3).

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` /
reference leg of `bench.py` may import, call or execute anything under `oracle/`. The product path
(the CUDA library and its Python binding) never does, and shares no code with it.

Plain numpy/scipy in float64, pixel-vectorised, no blocking or fusion beyond each definition.

Parity status of each function is stated in its module header.
"""
