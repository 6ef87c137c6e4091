"""Seeded synthetic choice-based LP instances (inputs only).

This package draws the random data of a choice-based LP under the generalized
attraction model: prices, capacities, the product-resource incidence and the
per-segment consideration sets with their attractions. It holds none of the
solution method's arithmetic and is shared by the CPU oracle, the tests and the
benchmark. Nothing here imports the oracle or the CUDA library.
"""
from .gam import (Instance, batch_base, batch_family, full_offer_demand, huge_gam, make_instance, mid_gam,
                  paper_shaped, period_rates, seeded_duals, tiny_mnl, warm_family)

__all__ = ["Instance", "make_instance", "tiny_mnl", "mid_gam", "huge_gam", "paper_shaped", "full_offer_demand",
           "seeded_duals", "batch_base", "batch_family", "period_rates", "warm_family"]
