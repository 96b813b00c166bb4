"""B300-native differentiable 3D Gaussian splatting mapping step.

The compute path is the C-ABI library ``libgs.so`` (hand-written CUDA for
sm_103a); ``paper_2606_30436_b300.gs`` is its thin Python binding.  Importing the
package itself loads nothing, so the synthetic-input module can be used on a
machine without the library.
"""
__all__ = ["gs", "scenes"]
