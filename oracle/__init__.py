"""Plain, slow, float64 CPU oracle for the extraction method of Li & Shen, "Improving Efficiency of
Iso-Surface Extraction on Implicit Neural Representations Using Uncertainty Propagation".

This package is TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the CUDA library never does, and it shares no code,
table or constant with the library.  Every function restates the paper's definitions in the
paper's order with numpy (matrix products are the only library primitive), so that each step can
be checked against the paper by eye.

Modules
  mlp      -- ReLU MLP evaluation (the INR of Sec. III-B, App. E).
  affine   -- affine forms and their rules (Sec. III-A, Eqs. 1-4), probabilistic affine forms with
              the CLT read-off and least-squares linearisation (Sec. IV-B, Eqs. 6-10, Table VII),
              the uniform-assumption read-off RA-UA (Sec. IV-A), and a covariance propagation
              used as an independent cross-check of the CLT sigma.
  octree   -- hierarchical culling of Algorithm 1, run level by level over octree cubes, and the
              dense ground truth (Sec. V-A.3).
  mc       -- a marching-cubes case table generated from first principles and marching cubes
              over a lattice of corner values (Sec. IV-D, last paragraph).
  proposer -- the small cell-subdivision MLP with a hand-written backward pass and BCE loss.
"""
