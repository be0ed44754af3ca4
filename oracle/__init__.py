"""Plain FP64 CPU reference (oracle) for the multigrid hot path.

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's CPU-baseline
leg to check and time the CUDA path.  Nothing in the product package imports it.
"""
