"""B300-native (sm_103a) differentiable tile rasterizer for 3D Gaussians with
the Gaussian Splashing underwater image-formation model folded into
compositing (arXiv 2411.19588, Sec. IV)."""
