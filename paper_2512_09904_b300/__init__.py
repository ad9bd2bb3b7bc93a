"""B300-native coupled fluid-solid-thermal SPH hot path (arXiv 2512.09904).

The compute path is the CUDA library libsph_b300.so (sm_103a) behind a C ABI;
`paper_2512_09904_b300.sph` is its thin ctypes binding.  `workloads` holds
the seeded synthetic inputs.
"""
