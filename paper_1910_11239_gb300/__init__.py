"""GB300-native fast tensor-product Schwarz smoothers for SIPG multigrid.

Implements the method of Witte, Arndt and Kanschat (fast diagonalization
local solvers inside geometric multigrid for the interior penalty DG
Laplacian on Cartesian meshes) as hand-written sm_103a CUDA behind the C ABI
of include/tpss.h.  ``tpss`` is the thin Python binding; ``build_lib`` builds
the library; ``workloads`` holds the seeded synthetic inputs; ``perf`` holds
the algorithmic flop/byte counts used for roofline reporting.
"""
