"""Batched SQP trajectory optimisation on GB300 (GATO, arXiv 2510.07625).

``paper_2510_07625_gb300.gato`` binds the C ABI of ``libgato.so`` (hand-written
sm_103a CUDA); ``paper_2510_07625_gb300.inputs`` draws the seeded workloads.
"""
