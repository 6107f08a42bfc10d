"""FP64 CPU oracle for the SE(2) convolution path.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU legs
of bench.py may import this package.  The CUDA product path never imports it.
"""
