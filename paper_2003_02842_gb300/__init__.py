"""GB300-native Malliavin-Mancino Fourier covariance estimator via type-1 NUFFTs."""
