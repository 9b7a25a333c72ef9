"""GB300-native sampler for the average spectrum method with blocked modes
sampling (Ghanem & Koch, arXiv:1912.01379).

paper_1912_01379_gb300.asm      -- binding of the C ABI (include/asm.h)
paper_1912_01379_gb300.build    -- in-tree nvcc build of libasm_gb300.so
paper_1912_01379_gb300.workloads -- seeded synthetic inputs
"""
__all__ = ["asm", "build", "workloads"]
