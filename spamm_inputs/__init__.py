"""Seeded synthetic matrices shared by the oracle and the CUDA path (no SpAMM
arithmetic here)."""
from .generators import (algebraic_decay, batched_products, exp_decay,  # noqa: F401
                         exp_decay_nonsym, hilbert_index_3d, normal,
                         poisson_arrivals, serving_requests, splitmix_u64,
                         uniform_dense, uniform_pm1, water_like,
                         water_like_sites)
