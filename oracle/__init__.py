"""FP64 CPU oracle of the FFT EnKF analysis step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method written from the paper (Mandel, Beezley, Kondratenko,
"Fast Fourier Transform Ensemble Kalman Filter with Application to a Coupled
Atmosphere-Wildland Fire Model").  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and it shares
no code, table or constant with the CUDA path.

Modules
  dft    explicit unitary 2-D DFT as dense DFT-matrix products (no FFT)
  enkf   eq. (dii) spectral variance, eq. (cov-multi-spectral) cross spectra,
         eq. (spectral-enkf) / (spectral-multi-enkf) update
  dense  brute-force forms used to pin the above on tiny grids: sample covariance
         C_N, diag(F C_N F*), and the dense EnKF update eq. (enkf) / (multi-enkf)
  sine   the real sine transform variant (Sec. 4): orthonormal DST-I on the interior nodes,
         boundary nodes unchanged
  mlp    FP64 forward/backward of the spectral-variance denoiser and its
         radial binning (not in the paper; parity of trained weights unpinned)

Readings of points the paper leaves open are stated where they are used:
unitary F; cross spectrum conjugated on the observed block; gain zero where
chat + rhat == 0; mutual cross-covariances of observed blocks neglected (Sec. 2.2).
"""
