"""GB300 library for the exact pressure elimination (algebraic hybridisation)
of the Crouzeix-Raviart P1-nonconforming / P0 Stokes and Navier-Stokes
systems (Chenier & Eymard, arXiv 2101.03777).

The computation runs in the CUDA library ``libcrhyb.so`` (C interface in
``include/crhyb.h``); ``crhyb`` is its Python binding.
"""

from .crhyb import (  # noqa: F401
    CrError,
    EXPORTED,
    LIB_PATH,
    cr_apply_G,
    cr_assemble_coupled,
    cr_hybrid_export,
    cr_hybridise,
    cr_mesh_face_elements,
    cr_mesh_faces,
    cr_mesh_load,
    cr_mesh_mis,
    cr_recover_up,
    cr_solve,
    ell_to_csr,
    load_library,
)
