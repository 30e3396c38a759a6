"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package holds no arithmetic of the DGSEM method itself: it lays out
periodic hexahedral meshes (equispaced geometry samples per element plus
face connectivity) and draws random nodal states from seeds.  Everything that
turns these inputs into a discretisation (LGL nodes, metrics, fluxes) lives
separately in the CUDA library and in the oracle.
"""
from .mesh import Mesh, box_mesh, ROTATIONS, face_node_flip  # noqa: F401
from .states import random_state, tgv_params, mms_params, ensemble_members  # noqa: F401
