"""GB300 (sm_103a) NSGA-III environmental selection (arXiv 2503.20286).

The computation lives in ``libemo.so`` (CUDA, C ABI declared in
``include/emo.h``); ``_binding`` marshals torch tensors to it. Importing the
package does not load CUDA; the binding functions load the library on first
use and raise when it is missing.
"""
__all__ = ["emo_dominance", "emo_nd_rank", "emo_nsga3_select", "emo_nsga3_select_batch",
           "emo_workspace_size", "emo_batch_workspace_size", "emo_workspace_status",
           "emo_set_spin_budget", "emo_status_string", "emo_version", "workloads", "build"]


def __getattr__(name):
    if name in ("workloads", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    if name.startswith("emo_") or name in ("SelectInfo", "SelectDebug", "EmoError", "EmoLibraryError", "lib"):
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
