"""GB300-native FFT Ensemble Kalman Filter analysis step (sm_103a CUDA behind a C ABI).

Method: Mandel, Beezley, Kondratenko, "Fast Fourier Transform Ensemble Kalman
Filter with Application to a Coupled Atmosphere-Wildland Fire Model", Sec. 2.1.

  abi        ctypes binding of include/fftenkf.h (same names as the C entry points)
  torch_api  convenience wrapper taking torch CUDA tensors (marshalling only)
  build      nvcc build of libfftenkf.so for sm_103a
"""

__all__ = ["abi", "torch_api", "build"]
