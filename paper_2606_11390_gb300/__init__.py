"""GB300-native differentiable tile-based Gaussian splatting (sm_103a)."""
