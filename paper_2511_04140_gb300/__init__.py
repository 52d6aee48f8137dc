"""libfalcon for GB300: lossless FP64/FP32 time-series compression on the GPU.

The CUDA library (``_build/libfalcon.so``, C-ABI declared in ``include/falcon.h``)
does all the work; ``falcon`` is its thin ctypes binding.  Import
``paper_2511_04140_gb300.falcon`` to load it (it is not loaded on package import,
so the input generators in ``synth`` stay usable on machines without a GPU).
"""
__all__ = ["falcon", "synth", "build"]
