"""CPU oracle for the local block-sparse product -- test infrastructure only.

Plain, slow, obviously correct FP64 statements of what the GPU library computes,
written from the paper's Sec. II (blocked CSR, block-pair products, stacks) and
Sec. III (densification). Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA library and never imports it.
"""
