"""GB300-native BatchLayout: force-directed graph layout with minibatch updates,
exact all-pairs or Barnes-Hut repulsion (Rahman, Sujon, Azad; arXiv 2002.08233).

The compute path is the CUDA library lib/libbatchlayout.so behind the C ABI in
include/batchlayout.h; ``core`` is its thin Python binding. Importing this
package loads nothing: the library is loaded on first use.
"""

__all__ = ["core", "synth", "build"]


def __getattr__(name):
    if name in ("Graph", "Layout", "Server", "layout_batch", "use_torch", "BatchLayoutError"):
        from . import core
        return getattr(core, name)
    raise AttributeError(name)
