"""GB300 (sm_103a) implementation of LiteVoxel's sparse-voxel rasterizer hot path.

The compute lives in ``liblitevoxel.so`` (C ABI: include/litevoxel.h), built
in-tree by :func:`paper_2511_02510_gb300.build.build`; ``litevoxel`` is the
thin ctypes binding and ``raster`` the workspace-managing wrapper.
"""
__all__ = ["build", "litevoxel", "raster", "synth"]
