"""GB300-native PNP-cDFT library (arXiv:1407.0674): FFT evaluation of the cDFT
excess chemical potentials and the relaxed Gummel loop on one GPU, behind the
C ABI of include/pnp.h.  ``pnp`` is the ctypes binding, ``build`` compiles the
CUDA library in-tree for sm_103a."""
