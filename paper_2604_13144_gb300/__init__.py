"""GB300 (sm_103a) MPS TE-PAI: CUDA kernels behind a C-ABI (include/tepai.h).

The binding lives in paper_2604_13144_gb300.tepai; build the library with
paper_2604_13144_gb300.build.build().
"""
