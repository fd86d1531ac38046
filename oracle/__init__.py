"""FP64 CPU oracle for the DFPT chi0 path of plane-wave full-frequency GW.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import or run anything in this
package.  It shares no code with the CUDA library (paper_2203_05623_gb300) and
never imports it; both take their inputs from the seeded generator in synth/.

Everything here is plain NumPy / SciPy in float64 / complex128 on full
(non-symmetrised) plane-wave spheres, written for a reader checking it against
the paper by eye:

  model.py    plane-wave spheres, FFT grid maps, the Kohn-Sham Hamiltonian
              (dense matrix and dual-space FFT application, Sec. 4.1)
  chi0.py     density response: sum over states (Adler-Wiser, Sec. 2.2),
              Sternheimer solves (Eq. sternheimer) + Eq. dfpt, the free-electron
              closed form, finite differences of the ground-state density,
              the dense symmetrised matrix chi0bar = v^1/2 chi0 v^1/2 (Sec. 2.1),
              the sum over spin channels of a spin-polarised system
  pdep.py     PDEP eigenpairs of chi0bar (Sec. 3) by dense diagonalisation and
              by a textbook block Davidson iteration
  lanczos.py  Lanczos chains (Eq. lanczos and the recurrence above it, Sec. 3)
              on P_c h P_c and chi0 in the PDEP basis at imaginary frequencies
  dyson.py    the Dyson step chibar = (1 - chi0bar)^-1 chi0bar in a basis (Sec. 2)
  g0.py       G0 Lanczos chains of the unprojected h for the short-range
              correlation integral (Eq. ISR, Eq. lanczos, Sec. 3)
  sigma.py    exchange self-energy <psi_i|Sigma_X|psi_i> (Eq. sigmacIR, Sec. 2)

Parity status of each function is stated in its module header.
"""
