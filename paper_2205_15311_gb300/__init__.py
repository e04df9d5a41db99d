"""GB300-native JaTAM classification: stochastic tile self-assembly of whole
genotype spaces on one GPU (libjatam.so, include/jatam.h).

``binding`` wraps the C ABI; ``workloads`` holds the seeded synthetic input
generators.  Importing the package loads nothing: the library is loaded on
first use and every call fails loudly if it has not been built.
"""
