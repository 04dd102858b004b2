"""B300-native (sm_103a) cryoSplat orthographic splatting path (placeholder; filled in)."""
