"""GB300-native sparsity-aware SpMM (the single-GPU hot path of SHIRO, arxiv 2512.20178).

``shiro``    -- ctypes binding of libshiro (C ABI in include/shiro.h), same entry-point names;
``autograd`` -- torch.autograd.Function with the hand-written backward;
``synth``    -- seeded synthetic inputs shaped like the paper's graphs.
"""
