"""Split exponential Euler for N-coupled diffusion-reaction systems on curvilinear grids, on GB300.

The compute path is the C-ABI library ``libsexpe.so`` (hand-written CUDA for
sm_103a, built in-tree by ``__graft_entry__.build()``); ``binding`` wraps it
with ctypes.  Importing this package loads nothing: the library is opened on
first use and a missing library is an error, never a fallback.
"""
