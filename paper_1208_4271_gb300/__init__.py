"""GB300 (sm_103a) implementation of the MINE statistics over many variable
pairs (Albanese et al. 2012, minerva/minepy): the characteristic matrix M and
MIC, MAS, MEV, MCN, computed by the CUDA library libgmine behind the C ABI of
include/gmine.h.  `gmine` is the Python binding; `workloads` draws the seeded
synthetic inputs."""
