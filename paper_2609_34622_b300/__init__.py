"""B300-native BMND denoiser: CUDA kernels for sm_103a behind a C ABI."""
