"""FP64 CPU oracle of the porous lattice Boltzmann step (test infrastructure
only; see ``oracle.py``)."""
