"""CPU FP64 oracle of the bonded-particle magneto-elastic rod model.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py.  The product path (paper_2603_27279_gb300)
never imports it.
"""
from .oracle import (Oracle, align_z, bond, bond_damped, contact_pair, ibm_phi, lbm_lattice,  # noqa: F401
                     quat_mul, richardson, rotate)
