"""CPU oracle for the TTN trajectory simulator of color-code circuits.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

Everything here is a plain, slow, obviously-correct restatement of the
method of arXiv 2511.05719 ("Color code thresholds under circuit-level noise
beyond the Pauli framework"), in float64 / complex128:

  colorcode    -- the triangular 6.6.6 color code (Sec. II.A, App. A.1)
  circuit      -- syndrome-extraction circuit with circuit-level noise
                  locations (Sec. III, Fig. 1)
  philox       -- Philox4x32-10 counter-based generator (Salmon et al., SC'11),
                  the uniform draws of every stochastic event
  channels     -- SRX (Eq. 1), AD (Eqs. 2-3) and their Pauli-twirled
                  approximations (Sec. IV.C)
  statevector  -- O1: exact quantum-trajectory sampling on a state vector
                  (Sec. III.C)
  densitymatrix-- O2: exact channel evolution of the density matrix
  decoder      -- concatenated minimum-weight perfect matching (App. A.2)
  ttn          -- O4: plain binary tree tensor network trajectories
                  (Sec. III.B, App. B) with numpy's QR/SVD

Parity status of each function is stated in its module header.
"""
