"""GB300-native MDP path planner (arXiv 2109.00857): CUDA build of transition
probabilities and rewards, and sparse value iteration, behind the C ABI of
include/mdp.h.  ``mdp`` is the ctypes binding; ``inputs`` the seeded synthetic
environments."""
from . import inputs  # noqa: F401

__all__ = ["inputs", "mdp"]
