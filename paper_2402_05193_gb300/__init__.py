"""GB300-native (sm_103a) compressible-flow RHS / TVD-RK3 library."""
