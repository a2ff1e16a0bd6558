"""Plain FP64 CPU oracle of the Hu-Zhang-Geng thermal lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline / reference arm to check and time the GPU library.
The product package never imports anything from here.
"""
