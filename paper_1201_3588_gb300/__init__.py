"""GB300-native Monte Carlo dust radiative transfer (Lucy / Bjorkman-Wood packages
through a grid of cubes and subcubes), after Siebenmorgen, Heymann & Kruegel,
"PAH in vectorized three dimensional Monte Carlo dust radiative transfer models".

Submodules: ``workloads`` builds synthetic models (numpy only); ``rt`` binds the CUDA
library ``librt_gb300.so`` through its C ABI and raises if the library is missing.
Neither is imported here, so model building works without the CUDA library.
"""
