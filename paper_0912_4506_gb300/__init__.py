"""GB300-native temporally-blocked 3D 7-point Jacobi (Wittmann, Hager, Wellein,
arXiv:0912.4506).  Importing the package loads nothing; the CUDA library is
loaded by the first call that needs it and raises if it is missing."""
