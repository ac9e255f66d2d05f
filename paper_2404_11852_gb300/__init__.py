"""GB300 (sm_103a) voxel-grid NeRF rendering with sparse radiance warping (SpaRW).

``cicero`` is the Python binding of the C ABI in ``include/cicero.h`` (libcicero.so);
``autograd`` wraps the FP32 renderer and its hand-written backward as a torch.autograd.Function.
Both are imported on demand so that ``build`` and ``scenes`` work without a GPU.
"""
__all__ = ["cicero", "autograd", "build"]
