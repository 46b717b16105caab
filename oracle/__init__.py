"""Oracle for the batched Berends-Giele recursion (TEST INFRASTRUCTURE ONLY).

``bg_oracle`` is the literal, generic-number-type Python statement of the
recursion of arXiv:2502.07060 Sec. 2.2 plus the tensor-form brute-force
diagram sum; ``coracle`` binds the plain C twin used for bulk parity and the
timed CPU baseline.  Only tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.
"""
