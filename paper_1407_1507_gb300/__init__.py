"""GB300-native k-mer counter built on the method of KMC 2 (arXiv 1407.1507).

Submodules (imported on demand, so importing the package loads nothing):

* ``kmc``   -- ctypes binding of libkmc.so (include/kmc.h), the CUDA path.
* ``build`` -- nvcc build of libkmc.so for sm_103a.
* ``synth`` -- seeded synthetic genomes and reads (input generator only).
"""
