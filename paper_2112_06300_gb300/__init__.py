"""GB300-native continuous collision detection: sweep-and-prune broad phase and
conservative FP64 interval-bisection narrow phase (Belgrod et al., "Time of
Impact Dataset for Continuous Collision Detection and a Scalable Conservative
Algorithm"), as hand-written sm_103a CUDA kernels behind a C ABI
(include/ccd.h).  `ccd` is the binding, `scenes` the seeded input generators,
`build` compiles the library."""
