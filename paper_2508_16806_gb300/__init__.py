"""GB300-native restarted PDHG linear-programming solver (CUDA, sm_103a)."""
