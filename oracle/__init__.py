"""CPU oracle for the local block-sparse product -- test infrastructure only.

Plain, slow, obviously correct FP64 statements of what the GPU library computes,
written from the paper's Sec. II (blocked CSR, block-pair products, stacks) and
Sec. III (densification). Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg and reference arm (``--impl reference``, the
oracle timed on the host cores) may import this package. It shares no code with
the CUDA library and never imports it.
"""
