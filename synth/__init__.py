"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

Holds none of the solver's arithmetic: only phantom images, data terms
D_L built from them, capacity fields S, and label DAGs.  Both the FP64
oracle and the CUDA solver consume what these functions return.
"""
from .phantoms import (  # noqa: F401
    Problem,
    dagmf_batch,
    dagmf_problem,
    diff_problem,
    hmf_problem,
    hmf_tree,
    ishikawa_chain,
    ishikawa_problem,
    potts2d_problem,
    potts3d_problem,
    random_dag,
    random_problem,
)
