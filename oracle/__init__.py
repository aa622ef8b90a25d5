"""FP64 CPU oracle for joint time-frequency scattering (JTFS).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call or
execute anything in this directory; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code, tables or
constants with the CUDA path: both sides derive everything from the paper
(Lostanlen & Han, "Musical Metamerism with Time-Frequency Scattering").

Modules:
  jtfs_oracle  -- the multirate JTFS, loss and gradient (FP64, torch CPU).
  bruteforce   -- the same definition by direct O(n^2) circular convolution
                  with time-domain filters built by explicit DFT sums; for
                  tiny inputs only.  It pins jtfs_oracle.
  reconstruct  -- the reconstruction variant of §2.3: coloured-noise
                  initialisation from the target's S1 and momentum descent
                  with a bold-driver step size.
"""
