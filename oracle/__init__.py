"""CPU oracle for classified range-domain matching (Revathy & Jayamohan, "Dynamic Domain
Classification for Fractal Image Compression").

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct CPU restatement of
the method, written from the paper. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import it. The CUDA library never calls it and
shares no code, table or constant with it.

Modules (each function cites the passage of the paper it follows):
  geometry  range partition, overlapping domains, 2x2 domain contraction, square isometries
            (Section 1, Section 2 and Table 1)
  dbc       differential box counting local fractal dimension (Section 3.1) and the class
            index derived from the fractal distance (Section 3.1, Eq. 2-3)
  pools     the per-range dynamic domain pool (Section 3, Section 3.1 Eq. 3)
  fit       least-squares contrast/brightness and the exact collage error of one candidate
            (Section 1: the intensity part of each map)
  match     exact best-match search over each range's pool (plain C, exact integers)
  decode    iterated application of the stored maps from an initial image (Section 1), its
            adjoint with respect to the per-range contrast and brightness, and PSNR (Table 4)

Parity status: every function is pinned by tests under tests/ (closed forms, library routines,
brute force, group laws, contractivity). The paper prints no worked example for any of them, so
no pin reproduces a value printed in the paper except the Table 1 geometry counts.
"""
