"""GB300-native distributed FastMNMF (block-diagonal FastMNMF, arXiv 2605.19388).

The compute path is the C-ABI library ``libdfmnmf.so`` (hand-written CUDA for
sm_103a); ``paper_2605_19388_gb300.dfmnmf`` is its thin ctypes binding.
"""
__all__ = ["dfmnmf", "synth"]
