"""GB300-native Monte Carlo dust radiative transfer after SOC (Juvela 2019,
arXiv:1812.06632): photon packages traced through regular or octree grids by
hand-written sm_103a CUDA kernels behind the C-ABI library ``libsoc.so``, with
int64 fixed-point absorption counters and an FP64 equilibrium-temperature
update.

``paper_1812_06632_gb300.inputs`` (synthetic clouds and tables) imports
without the CUDA library.  ``paper_1812_06632_gb300.soc`` is the Python
binding of the C-ABI; it raises if ``libsoc.so`` has not been built.
"""
