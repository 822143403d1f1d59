"""GB300 (sm_103a) dirty-imaging library: the data-parallel hot path of BLINK (arXiv 2505.15204).

The compute path is the CUDA library under ``csrc/`` behind the C ABI of ``include/blink.h``;
``blink`` is its thin Python binding and ``build`` compiles it in-tree.
"""
