"""B300 (sm_103a) el-ph coupling interpolation and RTA linewidths.

Python face of the C ABI in include/phoebe_gpu.h (libphoebe_gpu.so, built
in-tree by ``python -m paper_2111_14999_b300.build``).  The binding is loaded
on first use of any of its names and raises if the library is missing or
stale: there is no CPU fallback.
"""
_BINDING_NAMES = (
    "EXPORTED", "PREC_BF16", "PREC_BF16X3", "PREC_FP64", "PREC_SPLIT_BF16", "PREC_SPLIT_FP16", "PREC_SPLIT_TF32",
    "PREC_TF32", "LIB_PATH", "PhoebeGPU", "PhoebeGPUError", "RTAParams", "constants", "lib", "make_params",
    "version", "binding",
)


def __getattr__(name):
    if name in _BINDING_NAMES:
        import importlib
        binding = importlib.import_module(__name__ + ".binding")
        return binding if name == "binding" else getattr(binding, name)
    raise AttributeError(name)
