"""CPU oracle for the isogeometric CFIE boundary element method (test infrastructure).

This package is test infrastructure, not part of the product path: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.  It is a plain,
slow FP64 restatement of the method, written for checking by eye against the paper:

  * ``bspline``    -- B-splines by the Cox-de Boor recursion and NURBS patch maps (Sec. 3.1, 3.2);
  * ``space``      -- the spline spaces S^2_{p,m} and S^0_{p,m} on the patches (Sec. 3.3);
  * ``quadrature`` -- Gauss rules and the regularising transforms for touching element pairs
                      (the paper does not specify them; see the module header);
  * ``assemble``   -- Galerkin matrices M, V, K, K', W (Sec. 4.1-4.3) and right-hand sides;
  * ``fmm``        -- cluster tree, admissibility and the interpolated-kernel ("mode B") matrix that
                      the fast multipole method reproduces (Sec. 4.4);
  * ``solve``      -- dense LU and restarted GMRES (Sec. 5.1);
  * ``farfield``   -- far-field pattern of the computed density (Sec. 1, 2);
  * ``mie``        -- the Mie series for the unit sphere (closed form, not from the paper).

It shares no code with the CUDA path.  The only module both sides import is the seeded input
generator ``paper_2306_11324_gb300.inputs`` (geometry control nets, directions, random vectors).
"""
