"""GB300-native EAM lattice-list molecular dynamics (MISA-MD hot path).

Import ``paper_2107_07866_gb300.misa`` for the C-ABI binding (loads the CUDA
library), ``paper_2107_07866_gb300.synth`` for seeded synthetic inputs.
"""
