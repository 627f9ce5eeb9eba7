"""GB300 (sm_103a) ray traversal of compact constrained tetrahedral meshes,
after Aman, Demirci & Gudukbay, arXiv 2103.02309.

The public C ABI is include/tetmesh.h; `tetmesh` is its Python front end.
Importing `paper_2103_02309_gb300.tetmesh` loads the CUDA library and fails
loudly when it has not been built.
"""
__all__ = ["build", "tetmesh"]
